/*
 * libsph -- GB300 (sm_103a) implementation of the per-time-step particle interaction
 * sweep of the SPH fluid / rigid-body / heat / phase-transition method of
 * Fuchs, Meier, Wall, Cyron (arXiv:2103.07925).
 *
 * C ABI: plain pointers and sizes, no C++ types, no exceptions across the boundary.
 * Every call returns an sph_status; sph_last_error() gives a thread-local message.
 *
 * Ownership: the library copies every input array (the caller keeps its buffers);
 * output buffers are caller-allocated host memory unless stated otherwise.  One
 * scene (or batch) must be driven by one host thread at a time.
 *
 * Units are the caller's; the method is unit-free.  Positions and vectors always
 * carry three components, z = 0 in 2D.
 */
#ifndef SPH_H
#define SPH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* particle kinds: fluid particle i, rigid particle r of a body k, wall boundary particle b
 * (Sec. 3.1.2 and Sec. 3.3.4) */
#define SPH_FLUID 0
#define SPH_RIGID 1
#define SPH_WALL 2

#define SPH_MAX_MATERIALS 16

typedef enum {
  SPH_OK = 0,
  SPH_ERR_INVALID = -1,   /* bad argument or inconsistent input */
  SPH_ERR_OOM = -2,       /* device or host allocation failed */
  SPH_ERR_CUDA = -3,      /* a CUDA call failed (message in sph_last_error) */
  SPH_ERR_NONFINITE = -4, /* a NaN or Inf appeared in the particle state */
  SPH_ERR_TIMEOUT = -5,   /* a bounded device wait gave up */
  SPH_ERR_CAPACITY = -6   /* a fixed capacity (bodies, batch slots, memory cap) is exceeded */
} sph_status;

/* One material (phase).  Fluid phases use rho0, c (artificial speed of sound, Eq. eos),
 * eta (dynamic viscosity, Eq. momentum); every phase carries cp and kappa (Eq.
 * heat_equation).  A phase with transitions_to >= 0 turns into that material when its
 * temperature crosses T_transition (Sec. 3.6): a rigid phase melts above it, a fluid
 * phase solidifies below it.  latent_heat > 0 switches that pair of phases to the
 * enthalpy form of the apparent-capacity extension named in the paper's remark on
 * latent heat, with a mushy interval of width mushy_width around T_transition.
 *
 * Concentration (the paper's remark on chemically induced transitions): every fluid and
 * rigid phase carries a concentration C with dC/dt = (1/rho) div(D grad C), discretised
 * as the heat equation of Sec. 3.5 (Cleary and Monaghan) with diffusivity D in place of
 * kappa and no capacity; wall particles do not take part.  C_fixed (not NaN) holds the
 * concentration of a phase at that value at all times (a reservoir, the gastric juice of
 * Sec. 4.5).  transition_by = 1 makes transitions_to fire when the concentration crosses
 * C_transition instead of the temperature crossing T_transition (a rigid phase turns
 * fluid above it, a fluid phase turns rigid below it). */
typedef struct {
  int32_t kind;
  double rho0, c, eta, cp, kappa;
  double T_transition;
  int32_t transitions_to;
  double latent_heat, mushy_width;
  double diffusivity, C_transition, C_fixed;
  int32_t transition_by;  /* 0: temperature, 1: concentration */
} sph_material;

/* Scene parameters.
 *  dim              2 or 3
 *  dx, h            initial particle spacing and smoothing length (the paper uses h = dx)
 *  kernel_support   kappa of r_c = kappa h (3 for the quintic spline, Sec. 3.1.1)
 *  box_min/max      cell lattice extent (Sec. 3.2); periodic axes repeat with this period
 *  gravity          body force per unit mass b (fluid and bodies)
 *  dt_mode          0: dt_fixed;  1: Eq. timestepcond evaluated every step
 *  k_contact/d_contact  contact stiffness and damping of Eq. contactforce; <= 0 / < 0
 *                   select defaults k_c = m_r (0.22 / dt_ref)^2, d_c = 0.2 sqrt(k_c m_r / 2)
 *                   with dt_ref = 0.25 h / c_max and m_r the smallest rigid particle mass
 *  precision        64: FP64 everywhere; 32: FP32 pair sums with cell-relative positions,
 *                   FP64 body sums, orientation and diagnostics
 *  skin             Verlet skin (Sec. 3.2 combines Verlet and cell lists): neighbour lists
 *                   hold pairs closer than r_c + skin and are rebuilt (with the cell
 *                   binning) when some particle has moved more than skin / 2 since the last
 *                   rebuild, so every evaluation still sees exactly the pairs closer than
 *                   r_c.  0: rebuild every step.  Cells have edge >= r_c + skin.
 *  rebin_interval   with skin > 0: also rebuild at least every rebin_interval steps (0: no
 *                   forced rebuild)
 *  key_order        0: Morton order of cells;  1: row-major order (x fastest)
 *  cells_per_group  cells along x handled by one warp (0 = automatic; row-major only);
 *                   -1: the search takes windows of 32 consecutive (sorted) particles,
 *                   split where they cross into the next row of cells
 *  body_capacity    maximum number of bodies including those created by solidification
 *                   (0: initial count + 1024)
 *  src_*            optional moving Gaussian surface heat source (not in the paper; a heat
 *                   input for powder-bed scenes): power density src_power, radius
 *                   src_radius, centre src_origin + src_speed t, acting within src_depth
 *                   below src_ztop on phases that take part in a transition
 *  p_background     background pressure p_b of the transport-velocity formulation that
 *                   Sec. 3.3.2 applies (after Adami, Hu and Adams 2013): fluid particles
 *                   are advected with u~ = u^{n+1/2} + dt/2 a~, a~_i = -(p_b / m_i)
 *                   sum_j (V_i^2 + V_j^2) dW/dr e_ij, and the momentum equation gains
 *                   (1/m_i) sum_j (V_i^2 + V_j^2) 1/2 (A_i + A_j) . e_ij dW/dr with
 *                   A = rho u (u~ - u) (zero for wall and rigid particles).  0: off. */
typedef struct {
  int32_t dim;
  double dx, h, kernel_support;
  double box_min[3], box_max[3];
  int32_t periodic[3];
  double gravity[3];
  int32_t dt_mode;
  double dt_fixed;
  double k_contact, d_contact;
  int32_t precision;
  double skin;
  int32_t rebin_interval;
  int32_t key_order;
  int32_t cells_per_group;
  int32_t body_capacity;
  int32_t n_materials;
  const sph_material* materials;
  double src_power, src_radius, src_speed[3], src_origin[3], src_depth, src_ztop;
  double p_background;
} sph_params;

/* Particles (Sec. 3.1.2: phase, position, velocity, mass, density, temperature, body).
 * All arrays have n rows; vectors are n*3 doubles, row-major.
 *  density          fluid: initial value (recomputed by Eq. densum); rigid and wall:
 *                   the constant density that sets the particle volume V = m / rho
 *  material         index into sph_params.materials; the material's kind is the kind
 *  body             body id of rigid particles (0 .. k-1), ignored otherwise
 *  wall_velocity    prescribed velocity of wall particles (nullable: zero)
 *  wall_temperature prescribed (Dirichlet) temperature of wall particles, NaN =
 *                   adiabatic (nullable: all adiabatic)
 *  concentration    initial concentration C (nullable: zero; phases with C_fixed start
 *                   at C_fixed) */
typedef struct {
  int64_t n;  /* 1 .. 2^26 (a neighbour list entry holds the index in 26 bits) */
  const double *pos, *vel, *mass, *density, *temperature;
  const int32_t *material, *body;
  const double *wall_velocity, *wall_temperature;
  const double* concentration;
} sph_particles_in;

/* Rigid bodies (Sec. 3.4).  Mass, centre of mass and inertia are always derived from
 * the rigid particles (Eqs. procwise_centerofmass, procwise_inertia); quat (w,x,y,z)
 * is the initial orientation, vel and omega the initial linear and angular velocity. */
typedef struct {
  int32_t k;
  const double *quat, *vel, *omega;
} sph_bodies_in;

typedef struct sph_scene sph_scene;

/* Create a scene on the current CUDA device.  Copies the inputs, bins the particles,
 * derives body mass quantities and evaluates the initial accelerations (one full
 * evaluation at t = 0).  stream: a cudaStream_t or NULL (the library creates one).
 * Errors: SPH_ERR_INVALID (bad sizes, particle outside a non-periodic box, fewer than
 * three cells on a periodic axis, body without particles), SPH_ERR_OOM, SPH_ERR_CUDA. */
sph_status sph_create_scene(const sph_params* params, const sph_particles_in* particles,
                            const sph_bodies_in* bodies, void* stream, sph_scene** out);

/* Advance nsteps time steps of the velocity-Verlet scheme of Sec. 3.7 (asynchronous on
 * the scene's stream except for a final status read).  Errors after the steps ran:
 * SPH_ERR_NONFINITE if a fluid velocity went non-finite; SPH_ERR_CAPACITY if a phase
 * relabel (Sec. 3.6) needed more new bodies than body_capacity; SPH_ERR_TIMEOUT if the
 * bounded union-find hooking that groups solidifying particles into new bodies gave up.
 * In the last two cases that relabel is not applied (materials and body ids stay as they
 * were), and no later relabel of the scene is applied either. */
sph_status sph_step(sph_scene* scene, int32_t nsteps);

/* Same as sph_step without the final status read (no host synchronisation). */
sph_status sph_step_async(sph_scene* scene, int32_t nsteps);

/* field bits for sph_read_fields / sph_write_fields; dst[b] receives field bit b */
enum {
  SPH_F_POS = 0,   /* n*3 double */
  SPH_F_VEL = 1,   /* n*3 double: fluid u, rigid u_r, wall prescribed velocity */
  SPH_F_ACC = 2,   /* n*3 double: fluid acceleration a_i */
  SPH_F_RHO = 3,   /* n double */
  SPH_F_PRES = 4,  /* n double: fluid EOS pressure, wall/rigid extrapolated pressure */
  SPH_F_TEMP = 5,  /* n double: temperature (walls: prescribed value or NaN) */
  SPH_F_DTEMP = 6, /* n double: dT/dt (dH/dt for enthalpy phases) of the last evaluation */
  SPH_F_MAT = 7,   /* n int32 */
  SPH_F_BODY = 8,  /* n int32 (-1 for non-rigid) */
  SPH_F_FORCE = 9, /* n*3 double: f_r of rigid particles (Eq. rigidparticle_force) */
  SPH_F_VEXT = 10, /* n*3 double: extrapolated velocity of wall and rigid particles */
  SPH_F_CELL = 11, /* n int32: row-major cell index cx + nx (cy + ny cz) */
  SPH_F_ENTH = 12, /* n double: specific enthalpy (enthalpy phases) */
  SPH_F_BACC = 13, /* n*3 double: background acceleration a~ of fluid particles (p_background > 0) */
  SPH_F_CONC = 14, /* n double: concentration (walls: 0) */
  SPH_F_DCONC = 15, /* n double: dC/dt of the last evaluation */
  SPH_F_COUNT = 16
};

/* Copy fields to host.  original_order = 1 returns rows in input order, 0 in the
 * library's current (cell-sorted) order.  Synchronises the scene's stream. */
sph_status sph_read_fields(sph_scene* scene, uint32_t field_mask, void* const* host_dst,
                           int32_t original_order);

/* Post-processing (Eq. postprocessing): the Shepard-filtered field
 *   f^(r) = sum_j V_j f_j W(|r - r_j|) / sum_j V_j W(|r - r_j|)
 * at nq query points (host, nq*3 doubles; z ignored in 2D; wrapped on periodic axes) over
 * the particles whose material index i has bit i set in material_mask, closer than r_c.
 * field: SPH_F_VEL (3 values per query; walls contribute their prescribed velocity),
 * SPH_F_RHO, SPH_F_PRES, SPH_F_TEMP (walls: prescribed temperature) or SPH_F_CONC (1 value).
 * out: host, nq*3 or nq doubles, NaN where no particle contributes.  FP64 accumulation on
 * both paths.  Synchronises the scene's stream.  SPH_ERR_INVALID for other fields. */
sph_status sph_interpolate(sph_scene* scene, int64_t nq, const double* query, int32_t field,
                           uint32_t material_mask, double* out);

/* Overwrite POS, VEL and TEMP of fluid particles from host arrays in input order (FP64,
 * n rows of 3 or 1; rows of other particles are ignored).  Ownership stays with the
 * caller; the copy is enqueued on the scene's stream: a source in page-locked host memory
 * is read in place by the import kernel (keep it unchanged until the stream passes it, e.g.
 * until the next synchronising call), any other is staged before the call returns.  The
 * next step starts from the
 * written state with the accelerations of the last evaluation (its first half kick,
 * Sec. 3.7), as a staggered coupling with an outside solver does.  A written particle stays
 * in its cell frame: the Verlet-skin test of the next step decides whether the neighbour
 * lists are rebuilt; a particle written more than 64 cells away forces a rebuild.
 * SPH_ERR_INVALID for other fields or a null source of a requested field. */
sph_status sph_write_fields(sph_scene* scene, uint32_t field_mask, const void* const* host_src);

/* Body state (k rows; each pointer nullable): com k*3, quat k*4, vel k*3, omega k*3,
 * mass k, inertia k*9 (world frame), force k*3, torque k*3, alive k. */
typedef struct {
  double *com, *quat, *vel, *omega, *mass, *inertia, *force, *torque;
  int32_t* alive;
} sph_bodies_out;
sph_status sph_read_bodies(sph_scene* scene, const sph_bodies_out* out, int32_t* k_out);

/* FP64 diagnostics: [0..2] linear momentum, [3..5] angular momentum, [6] kinetic
 * energy, [7] thermal energy (sum m c_p T, or m H), [8] fluid+rigid mass, [9] time,
 * [10] step, [11] last dt, [12] fluid count, [13] rigid count, [14] live bodies,
 * [15] ordered pairs of the last force/heat sweep. */
sph_status sph_diagnostics(sph_scene* scene, double out[16]);

/* Neighbour sets N(a) = {b != a : |r_ab| < r_c} of the current positions, by input
 * index, ascending (test and export entry; FP64 scenes use the FP64 predicate).
 * counts: n int64; list: cap int32 (may be NULL to query the total). *total = sum. */
sph_status sph_neighbors(sph_scene* scene, int64_t* counts, int32_t* list, int64_t cap,
                         int64_t* total);

/* Scene information: [0] n, [1] fluid, [2] rigid, [3] wall, [4] bodies, [5] cells,
 * [6] cells x, [7] cells y, [8] cells z, [9] steps taken, [10] kernels per step,
 * [11] device bytes, [12] warp groups, [13] cells per group, [14] key order,
 * [15] ordered pairs evaluated by the force / heat sweep over all steps taken,
 * [16] neighbour-list rebuilds so far, [17] list capacity per particle, [18] particles that
 * changed phase so far, [19] threads per block of the pair sweeps, [20] blocks per SM of
 * the pair sweeps, [21] blocks per SM of the neighbour search.  out[] has 32 rows. */
sph_status sph_info(sph_scene* scene, int64_t out[32]);

/* Launch shape of the pair sweeps (density, extrapolation, force/heat) and of the
 * neighbour search, for autotuning.  cfg[0] threads per block of the sweeps (a multiple
 * of 32 in [32, 256]; default 256), cfg[1] resident blocks per SM of the sweeps and cfg[2]
 * of the search (0: as many as the occupancy allows; larger values are clamped to that).
 * n = number of entries given (missing entries take their defaults).  The shape changes
 * how work is spread over the GPU, never which arithmetic a particle sees: results are
 * bitwise the same for every shape.  SPH_ERR_INVALID on a bad shape. */
sph_status sph_set_launch(sph_scene* scene, const int32_t* cfg, int32_t n);
/* device time (ms, CUDA events on the scene's stream) of nsteps steps; the scene advances */
sph_status sph_time_steps(sph_scene* scene, int32_t nsteps, double* ms);

/* Tracing: run reps complete steps with the kernels launched one by one (no graph) and
 * CUDA events between them; ms_per_stage[SPH_PROFILE_STAGES] receives the mean device
 * time of each stage.  The scene advances by reps steps. */
#define SPH_PROFILE_STAGES 21
sph_status sph_profile(sph_scene* scene, int32_t reps, double* ms_per_stage);
const char* sph_profile_stage_name(int32_t stage);

void sph_destroy_scene(sph_scene* scene);
const char* sph_last_error(void);

/* ------------------------------------------------------------------ measured FP32 peak
 * A measurement aid (the paper has no counterpart): FP32 FMA throughput of the current
 * device, measured by a kernel of this library that runs independent FMA chains on every
 * SM (grid = 4 blocks of 256 threads per SM), timed with CUDA events on a stream of its own
 * (best of four launches after a warm-up).  iters: loop trips per thread (each trip is 128
 * FMA per thread); *tflops: 2 x FMA / s in 1e12; *sm_count (nullable): the device's SM
 * count; *ms (nullable): the best launch time.  It allocates and frees a small output
 * buffer.  Errors: SPH_ERR_INVALID (iters < 1 or tflops NULL), SPH_ERR_CUDA. */
sph_status sph_fp32_peak(int32_t iters, double* tflops, int32_t* sm_count, double* ms);

/* ------------------------------------------------------------------ allocation-free density
 * For callers that cannot allocate device memory: code running under a memory manager
 * that owns every device allocation, inside a region where allocation is not allowed, or
 * next to a framework that has taken the device memory.  (The paper has no counterpart;
 * this is a service of the library, not a step of the method.)
 *
 * Computes rho_i = m_i (W(0) + sum_j W_ij) over all j != i with |r_ij| < kernel_support h
 * (quintic spline, the density summation of the scene path) for n particles held in the
 * caller's device memory.  pos: device, n*3 doubles (z ignored in 2D); mass: device, n
 * doubles; rho: device output, n doubles; box_min/box_max: HOST arrays of 3 doubles that
 * contain every particle (non-periodic; particles outside are clamped to the edge cells).
 * The work is enqueued on stream (NULL: the default stream) and not synchronised.
 *
 * No device memory is allocated: the cell-list scratch is a fixed static device array of
 * this library (about 6 MB, held by every GPU that loads the library until exit).  Limits:
 * n <= SPH_STATIC_MAX_PARTICLES and at most SPH_STATIC_MAX_CELLS cells of edge >= r_c in
 * the box; larger inputs return SPH_ERR_CAPACITY without running.  The first call on a
 * device looks up the array's device address (once per device, with that device current),
 * so make that first call before any stream capture; the address is kept for the life of
 * the process, so do not call this after cudaDeviceReset on that device.  Every call uses
 * the same array and leaves its contents behind (the counters are cleared at the start of
 * each call): calls that overlap on the GPU, on different streams or threads, race and
 * must be serialised.  Particles of a cell are visited in index order: the result is the
 * same bit for bit on every call with the same input. */
#define SPH_STATIC_MAX_PARTICLES (1 << 18)
#define SPH_STATIC_MAX_CELLS (1 << 18)
sph_status sph_density_static(int32_t dim, int64_t n, const double* pos, const double* mass, double h,
                              double kernel_support, const double* box_min, const double* box_max,
                              double* rho, void* stream);

/* ------------------------------------------------------------------ batches and serving
 * A batch advances many independent scenes (jobs) together: every stage of a step is one
 * launch over all resident scenes, driven by a device table of scene offsets, and the
 * whole step is a captured CUDA graph.  Jobs are admitted while their device footprint
 * fits under hbm_cap_bytes and a slot is free; finished jobs are reported by poll and
 * their memory is released when they are read out. */
typedef struct sph_batch sph_batch;
typedef struct {
  const sph_params* params;
  const sph_particles_in* particles;
  const sph_bodies_in* bodies;
  int32_t nsteps_total;
} sph_job_desc;

sph_status sph_batch_create(int32_t capacity_scenes, size_t hbm_cap_bytes, int32_t precision,
                            void* stream, sph_batch** out);
/* footprint estimate of one job in bytes (device memory it would hold) */
sph_status sph_job_footprint(const sph_job_desc* job, size_t* bytes);
/* SPH_ERR_CAPACITY when the job does not fit now (no slot or over the memory cap) */
sph_status sph_batch_admit(sph_batch* batch, const sph_job_desc* job, int64_t* job_id);
/* advance every resident, unfinished job by up to nsteps (jobs stop at nsteps_total) */
sph_status sph_batch_step(sph_batch* batch, int32_t nsteps);
/* ids of jobs that finished since the last poll (n_done <= max_done): jobs that reached
 * nsteps_total, and failed jobs, which stop advancing: fluid velocities became non-finite,
 * or a relabel could not be applied (new bodies beyond the body capacity, or the bounded
 * union-find hooking gave up); sph_batch_job_state tells finished and failed apart.
 * Synchronises the batch's stream. */
sph_status sph_batch_poll(sph_batch* batch, int64_t* done_ids, int32_t max_done, int32_t* n_done);
/* *state: 0 advancing, 1 finished (reached nsteps_total), 2 failed (see sph_batch_poll) */
sph_status sph_batch_job_state(sph_batch* batch, int64_t job_id, int32_t* state);
sph_status sph_batch_read_fields(sph_batch* batch, int64_t job_id, uint32_t field_mask,
                                 void* const* host_dst);
sph_status sph_batch_job_diagnostics(sph_batch* batch, int64_t job_id, double out[16]);
/* release a job's device memory and slot */
sph_status sph_batch_release(sph_batch* batch, int64_t job_id);
/* [0] resident jobs, [1] resident particles, [2] bytes in use, [3] steps taken,
 * [4] jobs still advancing, [5] kernel launches per batch step (2D and 3D scenes
 * together), [6] ordered pairs evaluated by the force / heat sweep so far, summed over
 * the resident jobs */
sph_status sph_batch_info(sph_batch* batch, int64_t out[8]);
/* launch shape (as sph_set_launch) of the batch's 2D (dim 2) or 3D (dim 3) scenes */
sph_status sph_batch_set_launch(sph_batch* batch, int32_t dim, const int32_t* cfg, int32_t n);
/* device time (ms) of sph_batch_step(batch, nsteps), which it performs */
sph_status sph_batch_time_steps(sph_batch* batch, int32_t nsteps, double* ms);
void sph_batch_destroy(sph_batch* batch);

#ifdef __cplusplus
}
#endif
#endif
