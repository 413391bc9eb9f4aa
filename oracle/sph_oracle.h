/*
 * FP64 CPU oracle of the SPH fluid / rigid-body / heat-conduction method of
 * Fuchs, Meier, Wall, Cyron, "An SPH framework for fluid-solid and contact
 * interaction problems including thermo-mechanical coupling and reversible
 * phase transitions" (arXiv:2103.07925).
 *
 * TEST INFRASTRUCTURE.  This library exists to check the CUDA path.  Only the
 * test-suite, the smoke check and the timed CPU baseline of the benchmark may
 * load it; the product library never includes this header, never links this
 * code and shares no helper with it.
 *
 * Every function follows the paper's equations in the paper's order with
 * plain loops in double precision (compiled with -ffp-contract=off).  Readings
 * where the paper is silent are listed at the top of sph_oracle.c.
 */
#ifndef SPH_ORACLE_H
#define SPH_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_FLUID 0
#define ORC_RIGID 1
#define ORC_WALL 2
#define ORC_MAXMAT 32

typedef struct {
  int32_t kind;
  double rho0, c, eta, cp, kappa;
  double T_transition;
  int32_t transitions_to;
  double latent_heat, mushy_width;
  double diffusivity, C_transition, C_fixed; /* concentration (R16) */
  int32_t transition_by;                     /* 0 temperature, 1 concentration */
} orc_material;

typedef struct {
  int32_t dim;
  double dx, h, kernel_support;
  double box_min[3], box_max[3];
  int32_t periodic[3];
  double gravity[3];
  int32_t dt_mode;
  double dt_fixed;
  double k_contact, d_contact;
  int32_t n_materials;
  orc_material materials[ORC_MAXMAT];
  int32_t body_capacity;
  double src_power, src_radius, src_speed[3], src_origin[3], src_depth, src_ztop;
  double skin;         /* cells of the neighbour search have edge >= r_c + skin */
  int32_t force_brute; /* 1: brute-force O(N^2) neighbour search */
  double p_background; /* background pressure of the transport-velocity formulation (R15); 0: off */
} orc_params;

typedef struct orc_scene orc_scene;

/* field ids for orc_get */
enum {
  ORC_F_POS = 0, ORC_F_VEL, ORC_F_ACC, ORC_F_RHO, ORC_F_PRES, ORC_F_TEMP, ORC_F_DTEMP,
  ORC_F_MAT, ORC_F_BODY, ORC_F_FORCE, ORC_F_VEXT, ORC_F_CELL, ORC_F_ENTH, ORC_F_BACC, ORC_F_CONC, ORC_F_DCONC
};

orc_scene* orc_create(const orc_params* P, int64_t n, const double* pos, const double* vel,
                      const double* mass, const double* density, const double* temperature,
                      const int32_t* material, const int32_t* body, const double* wall_velocity,
                      const double* wall_temperature, int32_t k, const double* quat,
                      const double* bvel, const double* bomega, const double* concentration);
const char* orc_error(void);
int orc_step(orc_scene* s, int32_t nsteps);
void orc_get(orc_scene* s, int32_t field, void* out);
int64_t orc_n(orc_scene* s);
int32_t orc_nbodies(orc_scene* s);
/* bodies: com(k*3) quat(k*4) vel(k*3) omega(k*3) mass(k) inertia_world(k*9) force(k*3) torque(k*3) alive(k) */
void orc_get_bodies(orc_scene* s, double* com, double* quat, double* vel, double* omega,
                    double* mass, double* inertia, double* force, double* torque, int32_t* alive);
int64_t orc_neighbors(orc_scene* s, int64_t* counts, int32_t* list, int64_t cap);
void orc_diagnostics(orc_scene* s, double out[16]);
/* Shepard-filtered field at nq query points (Eq. postprocessing): field one of ORC_F_VEL,
 * ORC_F_RHO, ORC_F_PRES, ORC_F_TEMP, ORC_F_CONC; particles whose material bit is set in
 * material_mask contribute; out gets 3 (VEL) or 1 value per query, NaN without any
 * contributing particle within r_c.  Brute force over all particles.  Returns 0, or -1 for
 * an unsupported field. */
int orc_interpolate(orc_scene* s, int64_t nq, const double* query, int32_t field, uint32_t material_mask,
                    double* out);
void orc_destroy(orc_scene* s);

/* pieces exposed for pinning */
double orc_kernel_w(int32_t dim, double r, double h);
double orc_kernel_dw(int32_t dim, double r, double h);
void orc_body_mass_chunked(int32_t dim, double dx, int64_t n, const double* pos, const double* mass,
                           int64_t chunk, double* m_out, double* com_out, double* inertia_out);
void orc_quat_mul(const double* a, const double* b, double* out);
void orc_quat_rot(const double* q, double* R);

#ifdef __cplusplus
}
#endif
#endif
