/* npxo.c -- FP64 CPU oracle of the NeoPhysIx scene step.
 *
 * TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU-baseline leg are
 * the only callers.  It shares no code with the CUDA library and is written for a reader to
 * check against the paper by eye: one scene at a time, one point at a time, in double precision,
 * in the order the paper describes the step.
 *
 * Readings of the paper that this file fixes (the paper is silent on them):
 *  - z is up; the height map is indexed by the horizontal (x, y) (Sec. III-A); the friction
 *    least squares of Eqs. 1-6 is written in the horizontal plane, so its rotation alpha is yaw.
 *  - Cell index = floor((x - origin_x) * scale), clamped to the map (Sec. III-A says the
 *    coordinates are scaled by the factor and converted to integers).  That integer decision and
 *    the contact decision (point below the looked-up height) are taken in single precision, the
 *    precision of the GPU kernel, so that both sides decide the same integer from the same value.
 *  - Normal response (not described in the paper): a per-point penalty spring-damper along +z
 *    without adhesion, F_i = max(0, m_i (w_c^2 d_i - 2 zeta w_c vz_i)).
 *  - Integrator (not described): semi-implicit Euler on the CoG velocity and the world angular
 *    momentum, orientation advanced by the exponential map of the new angular velocity.
 *  - Joint angles (Sec. III-B): every K steps each angle is set to its clamped target; the robot
 *    stays one rigid body whose world CoG, root orientation and angular momentum are kept.
 *  - Friction (Sec. III-C): over the points in contact in both this and the previous step, the
 *    least-squares rigid map of Eq. 3 takes the points' positions after the step onto their
 *    positions before it; a3 ~ sin(alpha) (text below Eq. 6) is applied as an exact rotation by
 *    asin(a3) about the contact centroid.  Two such maps are solved: one for the slip caused by
 *    the joint motion (source: the points after the joint update, target: the step-start
 *    points), applied whole because the motors are strong enough (Sec. III-B), and one for the
 *    slip caused by the dynamics (source: the integrated points, target: the points before
 *    integration), scaled down so that its impulse never exceeds mu * (total normal force) * dt
 *    (the maximum static friction).  The CoG takes the scaled dynamic map, then the kinematic
 *    map; its velocity changes by the scaled dynamic displacement over dt, and the angular
 *    momentum by the yaw rate of the scaled dynamic rotation.
 *  - Two options (model fric_mode, off by default) follow the refinements the paper names after
 *    Eq. 6 without defining them: bit 0 weights every least-squares row by its point's normal
 *    force this step (the centroid becomes the centre of pressure; the Coulomb cap uses the
 *    force-weighted mean slip); bit 1 applies the dynamic correction's friction impulse
 *    J = M (v_new - v*) at the contact centroid, so that its torque about the CoG also turns the
 *    body about the horizontal axes (the x and y components of (centroid - CoG) x J; the vertical
 *    component stays the yaw of the least-squares rotation).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* The operation counter (opcount.h) exists only in the C++ counting build of this file; in the
 * plain build the region marks and the count of single-precision operations are empty. */
#ifdef NPXO_OPCOUNT
#include "opcount.h"
#else
#define NPXO_REGION(r) ((void)0)
#define NPXO_COUNT(kind, n) ((void)0)
#endif

#include "npxo.h"

#define NPXO_ACT_HOLD 0
#define NPXO_ACT_GP 2
#define NPXO_GP_LEN 32          /* program bytes (the 5-bit jump address reaches 32) */
#define NPXO_GP_PER_UPDATE 32   /* instructions executed per joint update */
#define NPXO_GP_KMAX 36         /* joint targets saturate at +-36 steps (+-180 degrees) */
#define NPXO_PI 3.14159265358979323846
#define NPXO_POINT_RADIUS 1e-3

/* ------------------------------------------------------------------ 3-vectors and 3x3 matrices */

static void mat_mul(const double A[9], const double B[9], double C[9]) {
    double T[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += A[3 * i + k] * B[3 * k + j];
            T[3 * i + j] = s;
        }
    memcpy(C, T, sizeof T);
}

static void mat_transpose(const double A[9], double B[9]) {
    double T[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) T[3 * j + i] = A[3 * i + j];
    memcpy(B, T, sizeof T);
}

static void mat_vec(const double A[9], const double x[3], double y[3]) {
    double t[3];
    for (int i = 0; i < 3; ++i) t[i] = A[3 * i] * x[0] + A[3 * i + 1] * x[1] + A[3 * i + 2] * x[2];
    memcpy(y, t, sizeof t);
}

/* inverse by the adjugate; returns 0 when the matrix is singular */
static int mat_inverse(const double A[9], double B[9]) {
    double c00 = A[4] * A[8] - A[5] * A[7];
    double c01 = A[5] * A[6] - A[3] * A[8];
    double c02 = A[3] * A[7] - A[4] * A[6];
    double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
    if (!(fabs(det) > 0.0)) return 0;
    double id = 1.0 / det;
    B[0] = c00 * id;
    B[1] = (A[2] * A[7] - A[1] * A[8]) * id;
    B[2] = (A[1] * A[5] - A[2] * A[4]) * id;
    B[3] = c01 * id;
    B[4] = (A[0] * A[8] - A[2] * A[6]) * id;
    B[5] = (A[2] * A[3] - A[0] * A[5]) * id;
    B[6] = c02 * id;
    B[7] = (A[1] * A[6] - A[0] * A[7]) * id;
    B[8] = (A[0] * A[4] - A[1] * A[3]) * id;
    return 1;
}

/* rotation by angle th about the unit axis u, right-hand rule (Rodrigues' formula) */
static void axis_angle(const double u[3], double th, double R[9]) {
    double c = cos(th), s = sin(th), k = 1.0 - c;
    R[0] = c + k * u[0] * u[0];        R[1] = k * u[0] * u[1] - s * u[2]; R[2] = k * u[0] * u[2] + s * u[1];
    R[3] = k * u[1] * u[0] + s * u[2]; R[4] = c + k * u[1] * u[1];        R[5] = k * u[1] * u[2] - s * u[0];
    R[6] = k * u[2] * u[0] - s * u[1]; R[7] = k * u[2] * u[1] + s * u[0]; R[8] = c + k * u[2] * u[2];
}

/* ------------------------------------------------------------------ quaternions (w, x, y, z) */

static void quat_to_mat(const double q[4], double R[9]) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* Hamilton product a (x) b */
static void quat_mul(const double a[4], const double b[4], double c[4]) {
    double t[4];
    t[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    t[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    t[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    t[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
    memcpy(c, t, sizeof t);
}

static void quat_normalize(double q[4]) {
    double n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int i = 0; i < 4; ++i) q[i] /= n;
}

/* unit quaternion of the rotation vector phi (angle |phi| about phi/|phi|) */
static void quat_from_rotvec(const double phi[3], double q[4]) {
    double a = sqrt(phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2]);
    if (a == 0.0) { q[0] = 1; q[1] = q[2] = q[3] = 0; return; }
    double s = sin(0.5 * a) / a;
    q[0] = cos(0.5 * a); q[1] = s * phi[0]; q[2] = s * phi[1]; q[3] = s * phi[2];
}

/* ------------------------------------------------------------------ model inputs */

typedef struct {
    int l0, nl, p0, np, j0;
    double *r;             /* [np*3] point offsets from the CoG in the shape frame */
    double *x0, *xp, *xs;  /* [np*3] world positions: step start, after joint update, after integration */
    unsigned char *kap;    /* [np] contact this step */
    double *F;             /* [np] normal force this step (0 out of contact) */
    double *wls;           /* [np] weights of the friction least-squares rows */
    double *Q, *T;         /* [nl*9], [nl*3] link frames (construction -> shape frame) */
    double Mtot, g[3], Ib[9], Ibinv[9];
    /* carried from the first half of a step to the second */
    double R[9], Iw_inv[9], om[3];
    int tick;
} scene_ws;

static int ws_alloc(scene_ws *w, int np, int nl) {
    w->r = (double *)malloc(sizeof(double) * 3 * (size_t)np);
    w->x0 = (double *)malloc(sizeof(double) * 3 * (size_t)np);
    w->xp = (double *)malloc(sizeof(double) * 3 * (size_t)np);
    w->xs = (double *)malloc(sizeof(double) * 3 * (size_t)np);
    w->kap = (unsigned char *)malloc((size_t)np);
    w->F = (double *)malloc(sizeof(double) * (size_t)np);
    w->wls = (double *)malloc(sizeof(double) * (size_t)np);
    w->Q = (double *)malloc(sizeof(double) * 9 * (size_t)nl);
    w->T = (double *)malloc(sizeof(double) * 3 * (size_t)nl);
    return w->r && w->x0 && w->xp && w->xs && w->kap && w->F && w->wls && w->Q && w->T;
}

static void ws_free(scene_ws *w) {
    free(w->r); free(w->x0); free(w->xp); free(w->xs); free(w->kap); free(w->F); free(w->wls);
    free(w->Q); free(w->T);
}

static void ws_bind(const npxo_model *M, int s, scene_ws *w) {
    w->l0 = M->link_off[s];
    w->nl = M->link_off[s + 1] - w->l0;
    w->p0 = M->point_off[s];
    w->np = M->point_off[s + 1] - w->p0;
    w->j0 = w->l0 - s;
}

static int max_scene_sizes(const npxo_model *M, int *np_max, int *nl_max) {
    *np_max = 1; *nl_max = 1;
    for (int s = 0; s < M->n_scenes; ++s) {
        int np = M->point_off[s + 1] - M->point_off[s];
        int nl = M->link_off[s + 1] - M->link_off[s];
        if (np < 1 || nl < 1) return -1;
        if (np > *np_max) *np_max = np;
        if (nl > *nl_max) *nl_max = nl;
    }
    return 0;
}

/* ------------------------------------------------------------------ Sec. III-B: joint angles */

/* Target angle of scene-local joint j at step n: bias + A sin(2 pi phase + phi).  The phase
 * advances by nu = round(f dt 2^32) / 2^32 turns per step and is taken modulo one turn in exact
 * integer arithmetic, so that it stays exact over long horizons. */
double npxo_target(const npxo_model *M, int scene, int jl, long long n) {
    const float *p = M->act_params + 4 * (size_t)(M->link_off[scene] - scene + jl);
    double A = p[0], f = p[1], phi = p[2], b = p[3];
    uint32_t nu = (uint32_t)(int64_t)llround((double)f * M->dt * 4294967296.0);
    uint32_t u = (uint32_t)((uint64_t)nu * (uint64_t)n);
    double turns = (double)u / 4294967296.0;
    return b + A * sin(2.0 * NPXO_PI * turns + phi);
}

/* ------------------------------------------------------------------ Sec. IV: GP controller */

/* Table I: an 8-bit opcode is a 3-bit command and a 5-bit value x.  000 move motor x left and 001
 * right (its target by -/+ one 5-degree step, saturating at +-NPXO_GP_KMAX steps; a motor the
 * scene lacks is ignored), 010 read sensor x (acc = foot-contact bit x of the last step), 011 load
 * x (acc = x), 100 jump to address x if acc != 0, 101 not (acc = ~acc), 110 inc, 111 dec.  The
 * accumulator is 8 bits wide (it wraps); the program counter wraps after the last address. */
void npxo_gp_run(const unsigned char *prog, unsigned char *pc, unsigned char *acc, signed char *k,
                 int nj, unsigned int sensors, int n_instr) {
    unsigned int p = *pc % NPXO_GP_LEN, a = *acc;
    for (int it = 0; it < n_instr; ++it) {
        const unsigned int op = prog[p] >> 5, x = prog[p] & 31u;
        unsigned int next = (p + 1) % NPXO_GP_LEN;
        switch (op) {
            case 0: if ((int)x < nj && k[x] > -NPXO_GP_KMAX) k[x] -= 1; break;
            case 1: if ((int)x < nj && k[x] < NPXO_GP_KMAX) k[x] += 1; break;
            case 2: a = (sensors >> x) & 1u; break;
            case 3: a = x; break;
            case 4: if (a != 0) next = x; break;
            case 5: a = ~a & 255u; break;
            case 6: a = (a + 1) & 255u; break;
            default: a = (a + 255u) & 255u; break;
        }
        p = next;
    }
    *pc = (unsigned char)p;
    *acc = (unsigned char)a;
}

/* Forward kinematics over the link tree, then the mass properties of the whole robot
 * (Sec. III-A: the mass points give the CoG and the momentum).  Each link's frame is its
 * parent's frame followed by the hinge rotation theta about the axis through the anchor, both
 * given in the parent's frame at rest (Appendix, createJoint). */
static void shape_update(const npxo_model *M, const npxo_state *st, scene_ws *w) {
    for (int l = 0; l < w->nl; ++l) {
        double *Q = w->Q + 9 * l, *T = w->T + 3 * l;
        int L = w->l0 + l;
        if (l == 0) {
            static const double I[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
            memcpy(Q, I, sizeof I);
            T[0] = T[1] = T[2] = 0.0;
            continue;
        }
        int P = M->parent[L];
        const double *QP = w->Q + 9 * P, *TP = w->T + 3 * P;
        double u[3] = {M->axis[3 * L], M->axis[3 * L + 1], M->axis[3 * L + 2]};
        double un = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        u[0] /= un; u[1] /= un; u[2] /= un;
        double a[3] = {M->anchor[3 * L], M->anchor[3 * L + 1], M->anchor[3 * L + 2]};
        double Rj[9], Ra[3], d[3];
        axis_angle(u, st->theta[w->j0 + l - 1], Rj);
        mat_mul(QP, Rj, Q);
        mat_vec(Rj, a, Ra);
        d[0] = a[0] - Ra[0]; d[1] = a[1] - Ra[1]; d[2] = a[2] - Ra[2];
        mat_vec(QP, d, T);
        T[0] += TP[0]; T[1] += TP[1]; T[2] += TP[2];
    }
    double Mt = 0.0, mp[3] = {0, 0, 0};
    for (int i = 0; i < w->np; ++i) {
        int I = w->p0 + i, l = M->plink[I];
        double p0[3] = {M->p0[3 * I], M->p0[3 * I + 1], M->p0[3 * I + 2]}, p[3];
        mat_vec(w->Q + 9 * l, p0, p);
        for (int k = 0; k < 3; ++k) {
            p[k] += w->T[3 * l + k];
            w->r[3 * i + k] = p[k];
            mp[k] += M->m[I] * p[k];
        }
        Mt += M->m[I];
    }
    w->Mtot = Mt;
    for (int k = 0; k < 3; ++k) w->g[k] = mp[k] / Mt;
    /* every mass point is a solid sphere of radius NPXO_POINT_RADIUS (2/5 m r^2 about any axis),
     * so that a single point or a line of points has an invertible inertia */
    memset(w->Ib, 0, sizeof w->Ib);
    for (int a = 0; a < 3; ++a) w->Ib[4 * a] = 0.4 * Mt * NPXO_POINT_RADIUS * NPXO_POINT_RADIUS;
    for (int i = 0; i < w->np; ++i) {
        double *r = w->r + 3 * i, m = M->m[w->p0 + i];
        for (int k = 0; k < 3; ++k) r[k] -= w->g[k];
        double rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) w->Ib[3 * a + b] += m * ((a == b ? rr : 0.0) - r[a] * r[b]);
    }
    mat_inverse(w->Ib, w->Ibinv);
}

/* ------------------------------------------------------------------ Sec. III-A: height map LUT */

static float lut_height(const npxo_model *M, int scene, double x, double y) {
    int hm = M->hmap[scene];
    if (hm < 0 || M->heightmaps == NULL) return 0.0f;
    float fx = ((float)x - (float)M->hm_origin[0]) * (float)M->hm_scale;
    float fy = ((float)y - (float)M->hm_origin[1]) * (float)M->hm_scale;
    NPXO_COUNT(NPXO_K_ADD, 2);   /* the single-precision subtractions and multiplications above */
    NPXO_COUNT(NPXO_K_MUL, 2);
    int ix = (int)floorf(fx), iy = (int)floorf(fy);
    if (ix < 0) ix = 0;
    if (ix > M->hm_nx - 1) ix = M->hm_nx - 1;
    if (iy < 0) iy = 0;
    if (iy > M->hm_ny - 1) iy = M->hm_ny - 1;
    return M->heightmaps[((size_t)hm * M->hm_ny + iy) * M->hm_nx + ix];
}

int npxo_lut(const npxo_model *M, int scene, double x, double y, double *h) {
    *h = lut_height(M, scene, x, y);
    return 0;
}

/* ------------------------------------------------------------------ Sec. III-C: friction LS */

/* Least-squares solution of Eqs. 4-6 for n point pairs (source s_i, residual e_i = target_i -
 * s_i), in coordinates centred on the source centroid: the translation t of the centred problem
 * and a3.  The paper's (a1, a2) equal t - a3 z x centroid.  With one point, or all points at one
 * place, the system is singular and a3 = 0 (translation only). */
int npxo_friction_ls(int n, const double *s, const double *e, double *t, double *a3) {
    double sb[2] = {0, 0}, eb[2] = {0, 0};
    t[0] = t[1] = 0.0;
    *a3 = 0.0;
    if (n < 1) return 0;
    for (int i = 0; i < n; ++i) {
        sb[0] += s[2 * i]; sb[1] += s[2 * i + 1];
        eb[0] += e[2 * i]; eb[1] += e[2 * i + 1];
    }
    sb[0] /= n; sb[1] /= n; eb[0] /= n; eb[1] /= n;
    double S2 = 0.0, X = 0.0;
    for (int i = 0; i < n; ++i) {
        double sx = s[2 * i] - sb[0], sy = s[2 * i + 1] - sb[1];
        S2 += sx * sx + sy * sy;
        X += sx * e[2 * i + 1] - sy * e[2 * i];
    }
    t[0] = eb[0]; t[1] = eb[1];
    if (n >= 2 && S2 > 1e-12) *a3 = X / S2;
    return 0;
}

/* The same least squares with row weights w_i >= 0 (the refinement the paper suggests after
 * Eq. 6: each term weighted by the force pressing its point against the ground): the weighted
 * centroid, t = the weighted mean residual, a3 = sum w (s~ x e) / sum w |s~|^2.  No weight: t = 0,
 * a3 = 0.  The rotation is solved when the weighted mean of |s~|^2 exceeds 1e-6 m^2 (a centre of
 * pressure spread over at least a millimetre; one point, or weight gathered on one point, gives a
 * translation only: the rotation is not determined there). */
int npxo_friction_ls_w(int n, const double *s, const double *e, const double *w, double *t, double *a3) {
    double W = 0.0, sb[2] = {0, 0}, eb[2] = {0, 0};
    t[0] = t[1] = 0.0;
    *a3 = 0.0;
    for (int i = 0; i < n; ++i) {
        W += w[i];
        sb[0] += w[i] * s[2 * i]; sb[1] += w[i] * s[2 * i + 1];
        eb[0] += w[i] * e[2 * i]; eb[1] += w[i] * e[2 * i + 1];
    }
    if (!(W > 0.0)) return 0;
    sb[0] /= W; sb[1] /= W; eb[0] /= W; eb[1] /= W;
    double S2 = 0.0, X = 0.0;
    for (int i = 0; i < n; ++i) {
        double sx = s[2 * i] - sb[0], sy = s[2 * i + 1] - sb[1];
        S2 += w[i] * (sx * sx + sy * sy);
        X += w[i] * (sx * e[2 * i + 1] - sy * e[2 * i]);
    }
    t[0] = eb[0]; t[1] = eb[1];
    if (S2 > 1e-6 * W) *a3 = X / S2;
    return 0;
}

/* weighted centroid of n horizontal points (w NULL: equal weights), the total weight and the
 * weighted spread sum w |s - centroid|^2 */
static void centroid_spread(int n, const double *s, const double *w, double *sb, double *W, double *S2) {
    sb[0] = sb[1] = 0.0;
    *W = 0.0;
    for (int i = 0; i < n; ++i) {
        const double wi = w ? w[i] : 1.0;
        *W += wi;
        sb[0] += wi * s[2 * i]; sb[1] += wi * s[2 * i + 1];
    }
    *S2 = 0.0;
    if (!(*W > 0.0)) return;
    sb[0] /= *W; sb[1] /= *W;
    for (int i = 0; i < n; ++i) {
        double dx = s[2 * i] - sb[0], dy = s[2 * i + 1] - sb[1];
        *S2 += (w ? w[i] : 1.0) * (dx * dx + dy * dy);
    }
}

/* the planar rigid map x -> centre + t + Rz(alpha) (x - centre) applied to the point x */
static void rigid_map_2d(const double centre[2], double tx, double ty, double alpha,
                         const double x[2], double out[2]) {
    double dx = x[0] - centre[0], dy = x[1] - centre[1];
    double ca = cos(alpha), sa = sin(alpha);
    out[0] = centre[0] + tx + ca * dx - sa * dy;
    out[1] = centre[1] + ty + sa * dx + ca * dy;
}

/* ------------------------------------------------------------------ one step of one scene */

/* First half of a step: step-start positions, the joint update, the positions after it and the
 * angular velocity (everything robot-robot contact reads). */
static void scene_pre(const npxo_model *M, npxo_state *st, int s, scene_ws *w, long long n,
                      npxo_counts *cnt) {
    double *c = st->c + 3 * s, *q = st->q + 4 * s, *L = st->L + 3 * s;
    const int np = w->np;
    double *R = w->R, *Iw_inv = w->Iw_inv, Rt[9], tmp[9];

    /* start-of-step world positions x = c + R r */
    NPXO_REGION(NPXO_R_SCENE);
    quat_to_mat(q, R);
    NPXO_REGION(NPXO_R_POINT);
    for (int i = 0; i < np; ++i) {
        double rw[3];
        mat_vec(R, w->r + 3 * i, rw);
        for (int k = 0; k < 3; ++k) w->x0[3 * i + k] = c[k] + rw[k];
    }

    /* Sec. III-B: every K steps the joints jump to their clamped targets; the robot stays one
     * rigid body whose CoG, orientation and angular momentum are kept */
    int tick = (M->act_mode != NPXO_ACT_HOLD) && (n % M->K == 0);
    w->tick = tick;
    NPXO_REGION(NPXO_R_TICK);
    if (tick) {
        int nj = w->nl - 1;
        /* the machine-code controller (Sec. IV): its instructions run, reading the foot contacts
         * of the last step, and set the targets in 5-degree steps */
        if (M->act_mode == NPXO_ACT_GP)
            npxo_gp_run(M->gp_prog + NPXO_GP_LEN * (size_t)s, st->gp_pc + s, st->gp_acc + s,
                        st->gp_k + w->j0, nj, st->sensors[s], NPXO_GP_PER_UPDATE);
        for (int j = 0; j < nj; ++j) {
            double th = M->act_mode == NPXO_ACT_GP ? st->gp_k[w->j0 + j] * (NPXO_PI / 36.0)
                                                   : npxo_target(M, s, j, n);
            double lo = M->lo[w->l0 + j + 1], hi = M->hi[w->l0 + j + 1];
            if (th < lo) th = lo;
            if (th > hi) th = hi;
            st->theta[w->j0 + j] = th;
        }
        shape_update(M, st, w);
        cnt->ticks += 1;
        cnt->tick_points += (unsigned long long)np;
        for (int i = 0; i < np; ++i) {
            double rw[3];
            mat_vec(R, w->r + 3 * i, rw);
            for (int k = 0; k < 3; ++k) w->xp[3 * i + k] = c[k] + rw[k];
        }
    } else {
        memcpy(w->xp, w->x0, sizeof(double) * 3 * (size_t)np);
    }

    /* angular velocity from the angular momentum: w = R Ib^-1 R^T L */
    NPXO_REGION(NPXO_R_SCENE);
    mat_transpose(R, Rt);
    mat_mul(R, w->Ibinv, tmp);
    mat_mul(tmp, Rt, Iw_inv);
    mat_vec(Iw_inv, L, w->om);
}

/* Second half: ground contact, integration with the external wrench fext (force, torque about the
 * CoG; NULL = none), friction, commit. */
static void scene_post(const npxo_model *M, npxo_state *st, int s, scene_ws *w, long long n,
                       double *ls_s, double *ls_e, npxo_counts *cnt, const double *fext) {
    double *c = st->c + 3 * s, *q = st->q + 4 * s, *v = st->v + 3 * s, *L = st->L + 3 * s;
    const double dt = M->dt;
    const int np = w->np;
    const int tick = w->tick;
    const double *Iw_inv = w->Iw_inv, *om = w->om;
    double tmp[9];
    (void)n;

    /* Sec. III-A: every mass point looks up the ground height under it; penalty normal force */
    const double kw2 = M->omega_c * M->omega_c, kc = 2.0 * M->zeta * M->omega_c;
    double FN = 0.0, tau[3] = {0, 0, 0};
    for (int i = 0; i < np; ++i) {
        const double *x = w->xp + 3 * i;
        NPXO_REGION(NPXO_R_POINT);
        float h = lut_height(M, s, x[0], x[1]);
        w->kap[i] = ((float)x[2] < h);
        w->F[i] = 0.0;
        if (!w->kap[i]) continue;
        NPXO_REGION(NPXO_R_CONTACT);
        double rho[3] = {x[0] - c[0], x[1] - c[1], x[2] - c[2]};
        double vz = v[2] + (om[0] * rho[1] - om[1] * rho[0]);
        double d = (double)h - x[2];
        double F = M->m[w->p0 + i] * (kw2 * d - kc * vz);
        if (F < 0.0) F = 0.0;
        w->F[i] = F;
        FN += F;
        tau[0] += rho[1] * F;
        tau[1] -= rho[0] * F;
        cnt->contacts += 1;
    }
    cnt->points += (unsigned long long)np;

    /* semi-implicit Euler */
    NPXO_REGION(NPXO_R_SCENE);
    double vs[3], Ls[3], cs[3], qs[4], oms[3], phi[3], dq[4], Rs[9];
    for (int k = 0; k < 3; ++k) vs[k] = v[k] + dt * M->gravity[k];
    vs[2] += dt * FN / w->Mtot;
    for (int k = 0; k < 3; ++k) Ls[k] = L[k] + dt * tau[k];
    if (fext)
        for (int k = 0; k < 3; ++k) {
            vs[k] += dt * fext[k] / w->Mtot;
            Ls[k] += dt * fext[3 + k];
        }
    mat_vec(Iw_inv, Ls, oms);
    for (int k = 0; k < 3; ++k) cs[k] = c[k] + dt * vs[k];
    for (int k = 0; k < 3; ++k) phi[k] = dt * oms[k];
    quat_from_rotvec(phi, dq);
    quat_mul(dq, q, qs);
    quat_normalize(qs);
    quat_to_mat(qs, Rs);

    /* Sec. III-C: friction over the contacts present in both steps */
    double cn[3] = {cs[0], cs[1], cs[2]}, vn[3] = {vs[0], vs[1], vs[2]}, Ln[3] = {Ls[0], Ls[1], Ls[2]};
    double qn[4] = {qs[0], qs[1], qs[2], qs[3]};
    /* friction model options: the least-squares rows weighted by their points' normal forces
     * (bit 0), and the friction impulse's torque about the horizontal axes (bit 1) -- the two
     * refinements the paper suggests after Eq. 6; 0 = Eqs. 1-6 as written */
    const int weighted = M->fric_mode & 1, tilt = M->fric_mode & 2;
    int nC = 0;
    double WC = 0.0;
    NPXO_REGION(NPXO_R_FRICTION);
    for (int i = 0; i < np; ++i)
        if (st->kappa[w->p0 + i] && w->kap[i]) { nC += 1; WC += weighted ? w->F[i] : 1.0; }
    if (nC >= 1 && WC > 0.0) {
        cnt->friction_pts += (unsigned long long)nC;
        /* dynamic slip: the map taking the integrated positions back onto the positions before
         * integration */
        double tD[2], a3D, sD[2], S2D, WD, zbar = 0.0;
        int k = 0;
        for (int i = 0; i < np; ++i) {
            if (!(st->kappa[w->p0 + i] && w->kap[i])) continue;
            double rw[3];
            mat_vec(Rs, w->r + 3 * i, rw);
            ls_s[2 * k] = cs[0] + rw[0];
            ls_s[2 * k + 1] = cs[1] + rw[1];
            ls_e[2 * k] = w->xp[3 * i] - ls_s[2 * k];
            ls_e[2 * k + 1] = w->xp[3 * i + 1] - ls_s[2 * k + 1];
            w->wls[k] = weighted ? w->F[i] : 1.0;
            zbar += w->wls[k] * (cs[2] + rw[2]);
            k++;
        }
        if (weighted) npxo_friction_ls_w(nC, ls_s, ls_e, w->wls, tD, &a3D);
        else npxo_friction_ls(nC, ls_s, ls_e, tD, &a3D);
        centroid_spread(nC, ls_s, weighted ? w->wls : NULL, sD, &WD, &S2D);
        zbar /= WD;
        /* kinematic slip (joint-update steps): the map taking the points moved by the joints
         * back onto their step-start positions */
        double tK[2] = {0, 0}, a3K = 0.0, sK[2] = {0, 0}, S2K = 0.0, WK = 0.0;
        if (tick) {
            k = 0;
            for (int i = 0; i < np; ++i) {
                if (!(st->kappa[w->p0 + i] && w->kap[i])) continue;
                ls_s[2 * k] = w->xp[3 * i];
                ls_s[2 * k + 1] = w->xp[3 * i + 1];
                ls_e[2 * k] = w->x0[3 * i] - w->xp[3 * i];
                ls_e[2 * k + 1] = w->x0[3 * i + 1] - w->xp[3 * i + 1];
                k++;
            }
            if (weighted) npxo_friction_ls_w(nC, ls_s, ls_e, w->wls, tK, &a3K);
            else npxo_friction_ls(nC, ls_s, ls_e, tK, &a3K);
            centroid_spread(nC, ls_s, weighted ? w->wls : NULL, sK, &WK, &S2K);
        }
        double aD = asin(a3D < -1 ? -1 : (a3D > 1 ? 1 : a3D));
        double aK = asin(a3K < -1 ? -1 : (a3K > 1 ? 1 : a3K));
        /* maximum static friction: the impulse that undoes the dynamic slip is at most
         * mu * FN * dt; beyond that the dynamic correction is scaled down */
        double sh = sin(0.5 * aD);
        double u2 = tD[0] * tD[0] + tD[1] * tD[1] + 4.0 * sh * sh * S2D / WD;
        double Jreq = w->Mtot * sqrt(u2) / dt;
        double Jmax = (double)M->mu[s] * dt * FN;
        double sc = (Jreq <= Jmax) ? 1.0 : Jmax / Jreq;
        /* CoG: first the scaled dynamic map about its centroid, then the kinematic map */
        double y[2], x2[2];
        rigid_map_2d(sD, sc * tD[0], sc * tD[1], sc * aD, cs, y);
        rigid_map_2d(sK, tK[0], tK[1], aK, y, x2);
        cn[0] = x2[0];
        cn[1] = x2[1];
        double yD[2];
        rigid_map_2d(sD, tD[0], tD[1], aD, cs, yD);
        vn[0] = vs[0] + sc * (yD[0] - cs[0]) / dt;
        vn[1] = vs[1] + sc * (yD[1] - cs[1]) / dt;
        double Rst[9], Iw[9], ez[3] = {0, 0, 1}, Iz[3];
        mat_transpose(Rs, Rst);
        mat_mul(Rs, w->Ib, tmp);
        mat_mul(tmp, Rst, Iw);
        mat_vec(Iw, ez, Iz);
        for (int k2 = 0; k2 < 3; ++k2) Ln[k2] = Ls[k2] + (sc * aD / dt) * Iz[k2];
        if (tilt) {
            /* the friction impulse J = M (v_new - v*) acts at the contact centroid (sD, zbar),
             * below the CoG: its torque about the CoG turns the body about the horizontal axes */
            const double Jx = w->Mtot * (vn[0] - vs[0]), Jy = w->Mtot * (vn[1] - vs[1]);
            const double rz = zbar - cs[2];
            Ln[0] += -rz * Jy;
            Ln[1] += rz * Jx;
        }
        double A = aK + sc * aD;
        double qz[4] = {cos(0.5 * A), 0.0, 0.0, sin(0.5 * A)};
        quat_mul(qz, qs, qn);
    }

    /* freeze a scene whose state is no longer finite or has left any sane range */
    NPXO_REGION(NPXO_R_SCENE);
    int bad = 0;
    for (int k = 0; k < 3; ++k) bad |= !isfinite(cn[k]) || !isfinite(vn[k]) || !isfinite(Ln[k]);
    for (int k = 0; k < 4; ++k) bad |= !isfinite(qn[k]);
    if (bad) { st->status[s] |= 1u; return; }
    if (fabs(vn[0]) > 1e3 || fabs(vn[1]) > 1e3 || fabs(vn[2]) > 1e3 ||
        fabs(cn[0]) > 1e6 || fabs(cn[1]) > 1e6 || fabs(cn[2]) > 1e6) {
        st->status[s] |= 2u;
        return;
    }
    memcpy(c, cn, sizeof cn); memcpy(v, vn, sizeof vn); memcpy(L, Ln, sizeof Ln); memcpy(q, qn, sizeof qn);

    /* contacts of this step become the previous contacts; foot sensors */
    unsigned int sens = 0;
    for (int i = 0; i < np; ++i) {
        st->kappa[w->p0 + i] = w->kap[i];
        int sid = M->sensor[w->l0 + M->plink[w->p0 + i]];
        if (w->kap[i] && sid >= 0 && sid < 32) sens |= 1u << sid;
    }
    st->sensors[s] = sens;
    cnt->scene_steps += 1;
    NPXO_REGION(NPXO_R_OTHER);
}

static void scene_step(const npxo_model *M, npxo_state *st, int s, scene_ws *w, long long n,
                       double *ls_s, double *ls_e, npxo_counts *cnt) {
    scene_pre(M, st, s, w, n, cnt);
    scene_post(M, st, s, w, n, ls_s, ls_e, cnt, NULL);
}

/* ------------------------------------------------------------------ robot-robot contact */

/* Robot-robot collision, named as future work after the API section: here every mass point is a
 * sphere of the given radius, and two points of different robots whose centres are closer than
 * two radii push each other apart along the line through their centres with the penalty law of
 * the ground contact (Sec. III-A's spring-damper, reading R4) written for the pair: stiffness
 * mu omega_c^2 and damping 2 zeta mu omega_c with mu = m_a m_b / (m_a + m_b) the pair's reduced
 * mass (so the pair's relative motion is a spring-damper of natural frequency omega_c), force
 * max(0, mu (omega_c^2 (2 r - d) - 2 zeta omega_c v_n)) with v_n the rate of change of d (a
 * force that is not a number counts as 0).  No friction acts between robots.  Every pair is
 * visited: no culling. */
void npxo_arena_forces(int n_robots, const int *np, const double *const *x, const float *const *m,
                       const double *c, const double *v, const double *om, const int *active,
                       double radius, double omega_c, double zeta, double *fext) {
    const double reach = 2.0 * radius, kw2 = omega_c * omega_c, kc = 2.0 * zeta * omega_c;
    for (int i = 0; i < 6 * n_robots; ++i) fext[i] = 0.0;
    for (int a = 0; a < n_robots; ++a) {
        if (!active[a]) continue;
        for (int b = 0; b < n_robots; ++b) {
            if (b == a || !active[b]) continue;
            for (int i = 0; i < np[a]; ++i) {
                const double *xi = x[a] + 3 * i;
                const double ri[3] = {xi[0] - c[3 * a], xi[1] - c[3 * a + 1], xi[2] - c[3 * a + 2]};
                /* velocity of the point: v + omega x r */
                const double *wa = om + 3 * a;
                const double vi[3] = {v[3 * a] + wa[1] * ri[2] - wa[2] * ri[1],
                                      v[3 * a + 1] + wa[2] * ri[0] - wa[0] * ri[2],
                                      v[3 * a + 2] + wa[0] * ri[1] - wa[1] * ri[0]};
                for (int j = 0; j < np[b]; ++j) {
                    const double *xj = x[b] + 3 * j;
                    const double d[3] = {xi[0] - xj[0], xi[1] - xj[1], xi[2] - xj[2]};
                    const double dist = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                    if (!(dist < reach) || dist == 0.0) continue;
                    const double nrm[3] = {d[0] / dist, d[1] / dist, d[2] / dist};
                    const double rj[3] = {xj[0] - c[3 * b], xj[1] - c[3 * b + 1], xj[2] - c[3 * b + 2]};
                    const double *wb = om + 3 * b;
                    const double vj[3] = {v[3 * b] + wb[1] * rj[2] - wb[2] * rj[1],
                                          v[3 * b + 1] + wb[2] * rj[0] - wb[0] * rj[2],
                                          v[3 * b + 2] + wb[0] * rj[1] - wb[1] * rj[0]};
                    const double vn = (vi[0] - vj[0]) * nrm[0] + (vi[1] - vj[1]) * nrm[1] + (vi[2] - vj[2]) * nrm[2];
                    const double ma = m[a][i], mb = m[b][j], mr = ma * mb / (ma + mb);
                    const double f = mr * (kw2 * (reach - dist) - kc * vn);
                    if (!(f > 0.0)) continue;   /* no adhesion; a force that is not a number (a robot
                                                   whose state went non-finite) exerts nothing */
                    const double F[3] = {f * nrm[0], f * nrm[1], f * nrm[2]};
                    double *o = fext + 6 * a;
                    o[0] += F[0]; o[1] += F[1]; o[2] += F[2];
                    o[3] += ri[1] * F[2] - ri[2] * F[1];
                    o[4] += ri[2] * F[0] - ri[0] * F[2];
                    o[5] += ri[0] * F[1] - ri[1] * F[0];
                }
            }
        }
    }
}

/* ------------------------------------------------------------------ public entry points */

static int check_model(const npxo_model *M) {
    if (M->n_scenes < 0 || M->K < 1 || !(M->dt > 0.0)) return -1;
    if (M->act_mode == NPXO_ACT_GP && !M->gp_prog) return -1;
    if (M->arena > 1 && (M->n_scenes % M->arena != 0 || !(M->arena_radius > 0.0) || !isfinite(M->arena_radius)))
        return -1;
    for (int s = 0; s < M->n_scenes; ++s) {
        int l0 = M->link_off[s], nl = M->link_off[s + 1] - l0;
        int p0 = M->point_off[s], np = M->point_off[s + 1] - p0;
        if (nl < 1 || np < 1) return -1;
        if (M->parent[l0] != -1) return -1;
        for (int l = 1; l < nl; ++l)
            if (M->parent[l0 + l] < 0 || M->parent[l0 + l] >= l) return -1;
        for (int i = 0; i < np; ++i)
            if (M->plink[p0 + i] < 0 || M->plink[p0 + i] >= nl || !(M->m[p0 + i] > 0.0f)) return -1;
    }
    return 0;
}

int npxo_init(const npxo_model *M, const float *origin, const float *quat, const float *vel,
              const float *omega, const float *theta0, npxo_state *st) {
    if (check_model(M)) return -1;
    int npm, nlm;
    if (max_scene_sizes(M, &npm, &nlm)) return -1;
    scene_ws w;
    if (!ws_alloc(&w, npm, nlm)) { ws_free(&w); return -2; }
    for (int s = 0; s < M->n_scenes; ++s) {
        ws_bind(M, s, &w);
        for (int j = 0; j < w.nl - 1; ++j) st->theta[w.j0 + j] = theta0[w.j0 + j];
        shape_update(M, st, &w);
        double q[4] = {quat[4 * s], quat[4 * s + 1], quat[4 * s + 2], quat[4 * s + 3]};
        quat_normalize(q);
        double R[9], Rt[9], tmp[9], Iw[9], Rg[3];
        quat_to_mat(q, R);
        mat_vec(R, w.g, Rg);
        for (int k = 0; k < 3; ++k) {
            st->c[3 * s + k] = origin[3 * s + k] + Rg[k];
            st->v[3 * s + k] = vel[3 * s + k];
        }
        for (int k = 0; k < 4; ++k) st->q[4 * s + k] = q[k];
        mat_transpose(R, Rt);
        mat_mul(R, w.Ib, tmp);
        mat_mul(tmp, Rt, Iw);
        double om[3] = {omega[3 * s], omega[3 * s + 1], omega[3 * s + 2]};
        mat_vec(Iw, om, st->L + 3 * s);
        for (int i = 0; i < w.np; ++i) st->kappa[w.p0 + i] = 0;
        st->sensors[s] = 0;
        st->status[s] = 0;
        if (st->gp_pc) { st->gp_pc[s] = 0; st->gp_acc[s] = 0; }
        if (st->gp_k)
            for (int j = 0; j < w.nl - 1; ++j) st->gp_k[w.j0 + j] = 0;
    }
    ws_free(&w);
    return 0;
}

/* Arenas: the robots of an arena advance in lock step, each step in two halves around their
 * contact forces, which all read the same step-start states.  A frozen robot takes no part. */
static int step_arenas(const npxo_model *M, npxo_state *st, int s0, int s1, int n_steps, long long step0,
                       npxo_counts *cnt) {
    const int A = M->arena;
    int npm, nlm;
    if (max_scene_sizes(M, &npm, &nlm)) return -1;
    if (s0 % A || s1 % A) return -1;
    scene_ws *ws = (scene_ws *)calloc((size_t)A, sizeof *ws);
    int *active = (int *)calloc((size_t)A, sizeof(int)), *np = (int *)calloc((size_t)A, sizeof(int));
    const double **x = (const double **)calloc((size_t)A, sizeof *x);
    const float **m = (const float **)calloc((size_t)A, sizeof *m);
    double *om = (double *)calloc(3 * (size_t)A, sizeof(double));
    double *fext = (double *)calloc(6 * (size_t)A, sizeof(double));
    double *ls_s = (double *)malloc(sizeof(double) * 2 * (size_t)npm);
    double *ls_e = (double *)malloc(sizeof(double) * 2 * (size_t)npm);
    int ok = ws && active && np && x && m && om && fext && ls_s && ls_e, nalloc = 0;
    for (; ok && nalloc < A; ++nalloc) ok = ws_alloc(&ws[nalloc], npm, nlm);
    if (ok) {
        for (int a0 = s0; a0 < s1; a0 += A) {
            for (int k = 0; k < A; ++k) {
                ws_bind(M, a0 + k, &ws[k]);
                shape_update(M, st, &ws[k]);
            }
            for (int t = 0; t < n_steps; ++t) {
                int any = 0;
                for (int k = 0; k < A; ++k) any |= (active[k] = st->status[a0 + k] == 0);
                if (!any) break;
                for (int k = 0; k < A; ++k) {
                    if (!active[k]) continue;
                    scene_pre(M, st, a0 + k, &ws[k], step0 + t, cnt);
                    np[k] = ws[k].np;
                    x[k] = ws[k].xp;
                    m[k] = M->m + ws[k].p0;
                    memcpy(om + 3 * k, ws[k].om, sizeof ws[k].om);
                }
                npxo_arena_forces(A, np, x, m, st->c + 3 * (size_t)a0, st->v + 3 * (size_t)a0, om, active,
                                  M->arena_radius, M->omega_c, M->zeta, fext);
                for (int k = 0; k < A; ++k)
                    if (active[k]) scene_post(M, st, a0 + k, &ws[k], step0 + t, ls_s, ls_e, cnt, fext + 6 * k);
            }
        }
    }
    if (ws)
        for (int k = 0; k < nalloc; ++k) ws_free(&ws[k]);
    free(ws); free(active); free(np); free(x); free(m); free(om); free(fext); free(ls_s); free(ls_e);
    return ok ? 0 : -2;
}

int npxo_step(const npxo_model *M, npxo_state *st, int s0, int s1, int n_steps, long long step0,
              npxo_counts *cnt) {
    if (M->arena > 1) return step_arenas(M, st, s0, s1, n_steps, step0, cnt);
    int npm, nlm;
    if (max_scene_sizes(M, &npm, &nlm)) return -1;
    scene_ws w;
    double *ls_s = (double *)malloc(sizeof(double) * 2 * (size_t)npm);
    double *ls_e = (double *)malloc(sizeof(double) * 2 * (size_t)npm);
    if (!ws_alloc(&w, npm, nlm) || !ls_s || !ls_e) { ws_free(&w); free(ls_s); free(ls_e); return -2; }
    for (int s = s0; s < s1; ++s) {
        ws_bind(M, s, &w);
        NPXO_REGION(NPXO_R_TICK);
        shape_update(M, st, &w);
        NPXO_REGION(NPXO_R_OTHER);
        for (int k = 0; k < n_steps; ++k) {
            if (st->status[s]) break;
            scene_step(M, st, s, &w, step0 + k, ls_s, ls_e, cnt);
        }
    }
    ws_free(&w);
    free(ls_s);
    free(ls_e);
    return 0;
}

typedef struct {
    const npxo_model *M; npxo_state *st; int s0, s1, n_steps; long long step0; npxo_counts cnt; int rc;
} npxo_job;

static void *npxo_worker(void *arg) {
    npxo_job *j = (npxo_job *)arg;
    memset(&j->cnt, 0, sizeof j->cnt);
    j->rc = npxo_step(j->M, j->st, j->s0, j->s1, j->n_steps, j->step0, &j->cnt);
    return NULL;
}

int npxo_step_mt(const npxo_model *M, npxo_state *st, int n_steps, long long step0, int n_threads,
                 npxo_counts *cnt) {
    /* threads take whole arenas */
    const int A = M->arena > 1 ? M->arena : 1, units = M->n_scenes / A;
    if (n_threads < 1) n_threads = 1;
    if (n_threads > units) n_threads = units > 0 ? units : 1;
    npxo_job *jobs = (npxo_job *)calloc((size_t)n_threads, sizeof *jobs);
    pthread_t *th = (pthread_t *)calloc((size_t)n_threads, sizeof *th);
    if (!jobs || !th) { free(jobs); free(th); return -2; }
    int rc = 0;
    for (int t = 0; t < n_threads; ++t) {
        memset(&jobs[t], 0, sizeof jobs[t]);
        jobs[t].M = M;
        jobs[t].st = st;
        jobs[t].s0 = A * (int)((long long)units * t / n_threads);
        jobs[t].s1 = A * (int)((long long)units * (t + 1) / n_threads);
        jobs[t].n_steps = n_steps;
        jobs[t].step0 = step0;
        if (pthread_create(&th[t], NULL, npxo_worker, &jobs[t])) { rc = -3; n_threads = t; break; }
    }
    for (int t = 0; t < n_threads; ++t) {
        pthread_join(th[t], NULL);
        if (jobs[t].rc) rc = jobs[t].rc;
        cnt->scene_steps += jobs[t].cnt.scene_steps;
        cnt->points += jobs[t].cnt.points;
        cnt->contacts += jobs[t].cnt.contacts;
        cnt->friction_pts += jobs[t].cnt.friction_pts;
        cnt->ticks += jobs[t].cnt.ticks;
        cnt->tick_points += jobs[t].cnt.tick_points;
    }
    free(jobs);
    free(th);
    return rc;
}

int npxo_points_world(const npxo_model *M, const npxo_state *st, int s, double *out) {
    int npm, nlm;
    if (max_scene_sizes(M, &npm, &nlm)) return -1;
    scene_ws w;
    if (!ws_alloc(&w, npm, nlm)) { ws_free(&w); return -2; }
    ws_bind(M, s, &w);
    shape_update(M, st, &w);
    double R[9];
    quat_to_mat(st->q + 4 * s, R);
    for (int i = 0; i < w.np; ++i) {
        double rw[3];
        mat_vec(R, w.r + 3 * i, rw);
        for (int k = 0; k < 3; ++k) out[3 * i + k] = st->c[3 * s + k] + rw[k];
    }
    ws_free(&w);
    return 0;
}

int npxo_mass_props(const npxo_model *M, const npxo_state *st, int s, double *g3, double *Ib9,
                    double *total_mass) {
    int npm, nlm;
    if (max_scene_sizes(M, &npm, &nlm)) return -1;
    scene_ws w;
    if (!ws_alloc(&w, npm, nlm)) { ws_free(&w); return -2; }
    ws_bind(M, s, &w);
    shape_update(M, st, &w);
    memcpy(g3, w.g, sizeof w.g);
    memcpy(Ib9, w.Ib, sizeof w.Ib);
    *total_mass = w.Mtot;
    ws_free(&w);
    return 0;
}

int npxo_link_frames(const npxo_model *M, const npxo_state *st, int s, double *out) {
    int npm, nlm;
    if (max_scene_sizes(M, &npm, &nlm)) return -1;
    scene_ws w;
    if (!ws_alloc(&w, npm, nlm)) { ws_free(&w); return -2; }
    ws_bind(M, s, &w);
    shape_update(M, st, &w);
    for (int l = 0; l < w.nl; ++l) {
        memcpy(out + 12 * l, w.Q + 9 * l, 9 * sizeof(double));
        memcpy(out + 12 * l + 9, w.T + 3 * l, 3 * sizeof(double));
    }
    ws_free(&w);
    return 0;
}

#ifdef NPXO_OPCOUNT
/* ------------------------------------------------------------------ the counting build's counters */
unsigned long long npxo_ops[NPXO_R_N][NPXO_K_N];
int npxo_region = NPXO_R_OTHER;

extern "C" void npxo_opcount_reset(void) {
    memset(npxo_ops, 0, sizeof npxo_ops);
    npxo_region = NPXO_R_OTHER;
}

/* out[r * NPXO_K_N + k]: operations of kind k counted in region r since the last reset */
extern "C" void npxo_opcount_get(unsigned long long *out) { memcpy(out, npxo_ops, sizeof npxo_ops); }
#endif
