/* npxo.h -- FP64 CPU oracle of the NeoPhysIx scene step (test infrastructure only).
 *
 * This is the checker, not the product: only the tests, the smoke check and the benchmark's
 * CPU-baseline leg load it.  It shares no code, header or constant with the CUDA library.
 *
 * One scene = one robot = one rigid body built from links of mass points (Sec. III-A, III-B);
 * links hang from their parent link by hinges (Appendix, createJoint).  The step follows
 * Sec. III in this order: joint-angle determination every K steps (III-B), point-cloud vs height
 * map collision (III-A), penalty normal forces, semi-implicit Euler integration, least-squares
 * friction correction (III-C, Eqs. 1-6), sensors.
 */
#ifndef NPXO_H
#define NPXO_H
#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int n_scenes;
    double dt, gravity[3];
    int K;                 /* joint-update interval in steps (Sec. III-B) */
    double omega_c, zeta;  /* per-point penalty spring: k = m omega_c^2, c = 2 zeta m omega_c */
    const int *link_off, *point_off;                     /* [S+1] */
    const float *p0, *m; const int *plink;                /* [P*3], [P], [P] */
    const int *parent; const float *anchor, *axis, *lo, *hi; const int *sensor; /* per link */
    const float *mu; const int *hmap;                     /* [S] */
    const float *heightmaps; int hm_nx, hm_ny; double hm_scale, hm_origin[2];
    int act_mode; const float *act_params;                /* [J*4]: A, f, phi, bias */
    int fric_mode;         /* bit 0: least-squares rows weighted by the normal forces; bit 1: the
                              friction impulse's torque about the horizontal axes (0 = Eqs. 1-6) */
    const unsigned char *gp_prog;  /* [S*32] machine-code programs (act_mode 2, Sec. IV, Table I) */
    int arena;             /* robots per arena (consecutive scenes sharing one ground and colliding
                              with one another; <= 1: every robot alone) */
    double arena_radius;   /* radius of the sphere around every mass point for robot-robot contact */
} npxo_model;

typedef struct {
    double *c, *q, *v, *L;       /* [S*3], [S*4] (w,x,y,z), [S*3], [S*3] world frame */
    double *theta;               /* [J] */
    unsigned char *kappa;        /* [P] contact flag of the previous step */
    unsigned int *sensors;       /* [S] foot-contact bits of the last step */
    unsigned int *status;        /* [S] 0 = ok, bit 0 non-finite, bit 1 out of bounds */
    unsigned char *gp_pc, *gp_acc;  /* [S] program counter and accumulator (act_mode 2) */
    signed char *gp_k;           /* [J] joint targets in 5-degree steps (act_mode 2) */
} npxo_state;

/* event counts: the numerators of the algorithmic-flop model */
typedef struct {
    unsigned long long scene_steps, points, contacts, friction_pts, ticks, tick_points;
} npxo_counts;

int  npxo_init(const npxo_model *M, const float *origin, const float *quat, const float *vel,
               const float *omega, const float *theta0, npxo_state *st);
int  npxo_step(const npxo_model *M, npxo_state *st, int s0, int s1, int n_steps,
               long long step0, npxo_counts *cnt);
int  npxo_step_mt(const npxo_model *M, npxo_state *st, int n_steps, long long step0,
                  int n_threads, npxo_counts *cnt);
int  npxo_points_world(const npxo_model *M, const npxo_state *st, int s, double *out_xyz);
int  npxo_mass_props(const npxo_model *M, const npxo_state *st, int s, double *g3, double *Ib9,
                     double *total_mass);
int  npxo_link_frames(const npxo_model *M, const npxo_state *st, int s, double *Q9t3);
double npxo_target(const npxo_model *M, int scene, int joint_local, long long n);
int  npxo_lut(const npxo_model *M, int scene, double x, double y, double *h);
int  npxo_friction_ls(int n, const double *src_xy, const double *e_xy, double *t2, double *a3);
int  npxo_friction_ls_w(int n, const double *src_xy, const double *e_xy, const double *w, double *t2,
                        double *a3);
/* Robot-robot contact forces at the given world positions (the future-work extension): robots
 * n_robots, robot k with np[k] points at x[k] ([np*3]), masses m[k], CoG c[k*3], velocity v[k*3],
 * angular velocity om[k*3]; active[k] = 0 leaves a robot out.  Writes the force and the torque
 * about the CoG on every robot to fext[k*6]. */
void npxo_arena_forces(int n_robots, const int *np, const double *const *x, const float *const *m,
                       const double *c, const double *v, const double *om, const int *active,
                       double radius, double omega_c, double zeta, double *fext);
/* The machine-code controller (Table I): n_instr instructions of prog from *pc, with accumulator
 * *acc, the scene's foot-contact bits `sensors` and the nj joint targets k (5-degree steps). */
void npxo_gp_run(const unsigned char *prog, unsigned char *pc, unsigned char *acc, signed char *k,
                 int nj, unsigned int sensors, int n_instr);

#ifdef __cplusplus
}
#endif
#endif
