/* npx.h -- C-ABI of the GB300 batched NeoPhysIx scene-step library (libnpx.so).
 *
 * A world holds many independent scenes; each scene is one robot made of links of mass points
 * (NeoPhysIx Sec. III-A) joined by hinges (Sec. III-B, Appendix "createJoint").  One call of
 * npx_world_step(w, n) advances every scene by n fixed steps on the GPU.  Each step:
 *   1. every K steps, joint-angle determination: each hinge jumps to its clamped target and the
 *      robot's shape is recomputed while it stays one rigid body (Sec. III-B);
 *   2. point-cloud collision: every mass point looks up the ground height under it in a height
 *      map (x, y scaled by the map's scale and floored to integer cells, Sec. III-A);
 *   3. a penalty normal force per point in contact, summed into the body wrench;
 *   4. semi-implicit Euler integration of the CoG and the angular momentum;
 *   5. friction estimation: the least-squares rigid correction of Eqs. 1-6 (Sec. III-C) over the
 *      points in contact in both steps, capped by the maximum static friction;
 *   6. foot-contact sensors.
 *
 * Conventions: SI units, z up, quaternions (w, x, y, z).  All arrays passed to the library are
 * HOST pointers unless a name says "device"; the library copies them during the call and never
 * keeps them.  Every function returns NPX_OK (0) or a negative NPX_E* code; npx_last_error()
 * then describes the failure (thread-local).  A world is not thread-safe: one caller thread at
 * a time.  Work is queued on the world's CUDA stream; functions that return data synchronise
 * that stream.
 */
#ifndef NPX_H
#define NPX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NPX_OK 0
#define NPX_EINVAL (-1)   /* bad argument (null pointer, index out of range, bad geometry) */
#define NPX_ENOMEM (-2)   /* host or device allocation failed */
#define NPX_ESTATE (-3)   /* call out of order (e.g. adding bodies after finalize) */
#define NPX_ECUDA (-4)    /* a CUDA runtime call failed */
#define NPX_ETIMEOUT (-5) /* a bounded device wait gave up */
#define NPX_ERANGE (-6)   /* a size exceeds what the library supports */

#define NPX_ACT_HOLD 0     /* joints keep their angles; no joint updates */
#define NPX_ACT_SINUSOID 1 /* target = bias + A sin(2 pi f t + phi), set every K steps */
#define NPX_ACT_GP 2       /* targets set by each scene's machine-code program (npx_gp_programs_set) */

/* Friction-model options (bits; 0 = the least squares of Sec. III-C, Eqs. 1-6, as written).  The
 * two refinements the paper names after Eq. 6: */
#define NPX_FRIC_WEIGHTED 1 /* every least-squares row weighted by its point's normal force */
#define NPX_FRIC_TILT 2     /* the friction impulse, applied at the contact centroid, also turns
                               the body about the horizontal axes */

#define NPX_MAX_LINKS 64         /* links per scene */
#define NPX_MAX_POINTS 2048      /* mass points per scene */
#define NPX_MAX_SENSORS 32       /* contact sensors per scene (one bit each) */

typedef struct npx_world npx_world;

/* World-wide parameters.  The height maps (Sec. III-A) are hm_count maps of hm_ny x hm_nx
 * float heights [m], row-major (row = y cell), cell (0,0) at world (hm_origin[0], hm_origin[1]),
 * hm_scale cells per metre (the paper's factor 10 gives 0.1 m cells).  A point at (x, y) reads
 * cell (floor((x - ox) * scale), floor((y - oy) * scale)) clamped to the map.  hm_count = 0
 * means flat ground z = 0 for every scene. */
typedef struct {
    int n_scenes;            /* number of scenes (>= 1) */
    float dt;                /* step [s] (> 0) */
    float gravity[3];        /* [m/s^2] */
    int joint_update_steps;  /* K: joints updated on steps n with n % K == 0 (Sec. III-B); >= 1 */
    float contact_omega;     /* per-point penalty natural frequency w_c [rad/s]: k = m w_c^2 */
    float contact_zeta;      /* per-point damping ratio: c = 2 zeta m w_c */
    int hm_count, hm_nx, hm_ny;
    float hm_scale;
    float hm_origin[2];
    const float *hm_data;    /* host, hm_count * hm_ny * hm_nx floats, or NULL when hm_count = 0 */
    void *stream;            /* cudaStream_t to queue work on (not the legacy default stream,
                                which cannot be captured); NULL = a stream the world creates */
    int device;              /* CUDA device ordinal */
} npx_world_desc;

/* Batched construction: scenes [first, first + count) in one call, structure of arrays.
 * Per scene s (0-based within the batch): links link_off[s] .. link_off[s+1]-1 and points
 * point_off[s] .. point_off[s+1]-1 of the arrays below.  Scene-local link 0 is the root; link
 * k >= 1 hangs from parent[k] < k by a hinge (scene-local joint k-1) through anchor[k] along
 * axis[k] (construction frame = the parent's frame with all angles zero, Appendix "createJoint"),
 * limited to [lo[k], hi[k]] rad.  sensor[k] >= 0 puts the link's points on contact sensor bit
 * sensor[k].  Points: construction-frame position p0 (xyz), mass m [kg] (> 0), scene-local link
 * plink.  mu[s] is the scene's friction coefficient, hmap[s] its height map (-1 = flat z = 0). */
typedef struct {
    int first, count;
    const int *link_off, *point_off;              /* [count + 1] */
    const int *parent;                            /* [n_links] */
    const float *anchor, *axis;                   /* [n_links * 3] */
    const float *lo, *hi;                         /* [n_links] */
    const int *sensor;                            /* [n_links] */
    const float *p0, *m;                          /* [n_points * 3], [n_points] */
    const int *plink;                             /* [n_points] */
    const float *mu;                              /* [count] */
    const int *hmap;                              /* [count] or NULL (all flat / map 0) */
} npx_scene_batch;

/* State and sensor read-out, all host arrays, any may be NULL. */
typedef struct {
    float *cog;        /* [S*3] world CoG */
    float *quat;       /* [S*4] orientation of the construction (root-link) frame */
    float *vel;        /* [S*3] CoG velocity */
    float *omega;      /* [S*3] world angular velocity */
    float *angmom;     /* [S*3] world angular momentum about the CoG */
    float *theta;      /* [J]   joint angles, scene-major (joint j of scene s at joint_off(s)+j) */
    uint32_t *contacts;/* [S]   contact-sensor bits of the last step */
    uint32_t *status;  /* [S]   0 = ok; bit 0 non-finite state, bit 1 out of range, bit 2 a
                                  height-map window copy that gave up its wait (scene frozen) */
    int64_t *step;     /* [1]   global step counter n */
} npx_sensors;

/* --- lifetime ------------------------------------------------------------------------- */
int npx_world_create(const npx_world_desc *desc, npx_world **out);
int npx_world_destroy(npx_world *w);
const char *npx_last_error(void);

/* --- construction, the paper's robot API (Sec. IV, Appendix) --------------------------- */
/* createPoint/createBox/...: a body is a cloud of n mass points (construction frame) of masses
 * mass[i], or of total_mass spread evenly when mass == NULL.  Returns the scene-local body id. */
int npx_body_add_pointcloud(npx_world *w, int scene, const float *xyz, const float *mass,
                            float total_mass, int n, int *out_body);
/* connectBodies: glue body2 rigidly to body1 (same link). */
int npx_body_connect(npx_world *w, int scene, int body1, int body2);
/* createJoint: hinge between the links of body1 (parent side) and body2, anchor in the
 * construction frame of body1, axis direction (normalised by the library), limits [lo, hi]. */
int npx_joint_add(npx_world *w, int scene, int body1, int body2, const float anchor[3],
                  const float axis[3], float lo, float hi, int *out_joint);
/* foot-contact sensor: bit `bit` is set when any point of the body's link touches the ground */
int npx_sensor_add(npx_world *w, int scene, int body, int bit);
int npx_scene_set_friction(npx_world *w, int scene, float mu);
int npx_scene_set_heightmap(npx_world *w, int scene, int hm);
/* copy scene src's construction into scenes [first_dst, first_dst + count) */
int npx_scene_clone(npx_world *w, int src, int first_dst, int count);
/* batched construction of many scenes at once (see npx_scene_batch) */
int npx_scenes_add(npx_world *w, const npx_scene_batch *b);
/* finalizeConstruction: checks every scene, packs the structure-of-arrays device layout,
 * uploads it.  All scenes must be defined.  Initial state: every scene at its construction pose
 * (origin 0, identity orientation, angles 0), at rest. */
int npx_world_finalize(npx_world *w);

/* --- state ------------------------------------------------------------------------------ */
/* Set every scene's pose and motion: construction-frame origin [S*3] and orientation [S*4]
 * (the paper's moveBody/rotateBody applied to the whole robot), CoG velocity [S*3], world
 * angular velocity [S*3], joint angles [J] (NULL keeps them).  Contact history is cleared. */
int npx_state_set(npx_world *w, const float *origin, const float *quat, const float *vel,
                  const float *omega, const float *theta);
/* Overwrite the whole dynamic state: CoG [S*3], orientation [S*4], CoG velocity [S*3], world
 * angular momentum about the CoG [S*3], joint angles [J], contact flags of the previous step per
 * mass point [P] (NULL clears them; 1 = in contact), and the global step counter n (which fixes
 * the joint-update phase n % K and the actuator phase).  Status words are cleared; the contact
 * sensors are recomputed from contact_prev.  The arrays are read before the call returns (each is
 * copied to the device once; pinned host memory makes that a DMA transfer). */
int npx_state_write(npx_world *w, const float *cog, const float *quat, const float *vel,
                    const float *angmom, const float *theta, const uint8_t *contact_prev,
                    int64_t step);
/* Per mass point contact flag of the last step [P] (1 = in contact), scene-major, in the order the
 * points were given; returns when the array is filled. */
int npx_contacts_read(npx_world *w, uint8_t *contact, size_t n);
/* Actuators: NPX_ACT_HOLD (params ignored) or NPX_ACT_SINUSOID with params [J*4] =
 * (amplitude rad, frequency Hz, phase rad, bias rad) per joint.  The phase advances by
 * round(f dt 2^32) / 2^32 turns per step (exact over any horizon). */
int npx_actuator_set(npx_world *w, int mode, const float *params);
/* The machine-code controller of Sec. IV (Table I) drives every scene's joints: programs [S*32]
 * (host), one 32-byte program per scene, each byte an opcode (upper 3 bits) and value x (lower 5):
 * 000 / 001 move motor x left / right (its target by -/+ 5 degrees, saturating at +-36 steps;
 * motors the scene lacks are ignored), 010 accumulator = foot-contact bit x of the last step,
 * 011 accumulator = x, 100 jump to address x if the accumulator is non-zero, 101 not, 110 inc,
 * 111 dec (8-bit accumulator; the program counter wraps after address 31).  At every joint
 * update (n % K == 0) each scene executes 32 instructions from its saved program counter, then
 * its joints take the clamped targets.  The call resets the program counters, accumulators and
 * targets (5-degree steps, 0 = the rest pose) and switches the world to NPX_ACT_GP; the state
 * blob carries the controller state; npx_actuator_set switches back. */
int npx_gp_programs_set(npx_world *w, const uint8_t *programs);
/* Controller state (host arrays, NULL to skip): program counters and accumulators [S], joint
 * targets in 5-degree steps [J] (write: each within +-36). */
int npx_gp_state_read(npx_world *w, uint8_t *pc, uint8_t *acc, int8_t *k);
int npx_gp_state_write(npx_world *w, const uint8_t *pc, const uint8_t *acc, const int8_t *k);
/* Friction model of the following steps: a combination of NPX_FRIC_* bits (0 by default).
 * NPX_FRIC_WEIGHTED: the least-squares centroid, moments and slip are weighted by the points'
 * normal forces of the step (the centroid becomes the centre of pressure); a rotation is solved
 * when the weighted mean squared spread about it exceeds 1e-6 m^2.  NPX_FRIC_TILT: the angular momentum
 * also changes by the x and y components of r x J, J = M dv the dynamic correction's impulse and r
 * the contact centroid relative to the CoG.  Unknown bits: NPX_EINVAL. */
int npx_world_set_friction_model(npx_world *w, int flags);
/* Robot-robot collision (the extension the paper names as future work, after its API section).
 * Scenes [a*size, (a+1)*size) form arena a: its robots share the ground and collide.  Every mass
 * point is a sphere of `radius` metres; two points of different robots of an arena whose centres
 * are closer than 2 radius push apart along the line through them with the ground contact's
 * penalty law for the pair (stiffness m_r w_c^2 and damping 2 zeta m_r w_c of the world's w_c and
 * zeta, m_r = m_a m_b / (m_a + m_b)); no friction acts between robots and the foot sensors report
 * ground contact only.  The forces are taken at the step's start (after the joint update) and
 * enter the integration with the ground forces; a frozen robot takes no part.
 * size: 1 (off, the default), 2 or 4, dividing the scene count; each arena runs in one warp, so
 * at most 32 / size lanes per scene (the call narrows the launch shape if needed; NPX_ERANGE when
 * the largest scene holds more than 64 * 32 / size points).  The learned surrogate refuses
 * worlds with arenas (NPX_EINVAL).  Errors: NPX_EINVAL for another size, a size that does not
 * divide the scene count, or radius <= 0 or not finite. */
int npx_world_set_arenas(npx_world *w, int size, float radius);
/* Advance all scenes n >= 0 steps (asynchronous on the world's stream). */
int npx_world_step(npx_world *w, int n);
/* Wait for queued work; reports a latched error of an earlier asynchronous call. */
int npx_world_sync(npx_world *w);
/* Fill the caller's arrays of npx_sensors (after the queued steps); returns when they are filled.
 * Each array is one copy from the device (pinned host memory makes it a DMA transfer). */
int npx_sensors_read(npx_world *w, npx_sensors *out);
/* World positions of one scene's mass points [n*3] (n = its point count) */
int npx_points_read(npx_world *w, int scene, float *xyz, int n);

/* --- checkpoint --------------------------------------------------------------------------- */
/* Serialise the dynamic state (state, angles, contact history, sensors, status, step counter)
 * into blob.  Call with blob == NULL to get the size. */
int npx_state_export(npx_world *w, void *blob, size_t *size);
int npx_state_import(npx_world *w, const void *blob, size_t size);

/* --- introspection and tuning -------------------------------------------------------------- */
typedef struct {
    int n_scenes, n_links, n_joints, n_points, max_points, max_links;
    int lanes_per_scene, warps_per_block, blocks, chunk_steps;
    int64_t step;
    int64_t kernel_launches;    /* step-kernel launches so far */
    int size_classes;           /* launches per chunk: scenes grouped by point count, each with
                                   its own shared-memory slots and launch shape */
    int hm_window_tma;          /* 1: each scene's 16 x 16-cell height-map window is loaded by
                                   one TMA box copy; 0: by plain loads (no maps, maps narrower or
                                   shorter than 16 cells, or rows not a multiple of 16 bytes) */
} npx_world_info;
int npx_world_info_get(npx_world *w, npx_world_info *out);
/* Launch shape of the step kernel: lanes per scene (4, 8, 16 or 32; a scene holds at most 64
 * points per lane), warps per block (1..16; shapes whose registers do not fit on an SM are refused
 * with NPX_ERANGE), resident blocks (0 = as many as fit), steps per kernel launch (chunk).  0 keeps
 * a value. */
int npx_world_configure(npx_world *w, int lanes_per_scene, int warps_per_block, int blocks,
                        int chunk_steps);
/* Time the step kernel over the feasible launch shapes on a copy of the state (n_steps each)
 * and keep the fastest; the world's state is unchanged.  Writes the chosen shape to *out. */
int npx_world_autotune(npx_world *w, int n_steps, npx_world_info *out);
/* Capture world_step's chunk sequence in CUDA graphs (1, default) or launch directly (0). */
int npx_world_use_graphs(npx_world *w, int on);
/* The step kernel's bounded wait for height-map window copies on its own, for tests of its failure
 * path: one warp whose 8-lane groups wait on mbarriers, two armed for a copy that is never issued
 * and two completed at once.  The wait gives up after its one-second limit; a step kernel whose
 * window copy gave up freezes the scene with status bit 2.  Synchronous: *gave_up (host) = lanes
 * whose wait gave up (16 expected), *completed = lanes that saw their barrier complete (16),
 * *elapsed_us = how long the wait took; the context stays usable. */
int npx_window_wait_selftest(int *gave_up, int *completed, int *elapsed_us, void *stream);

/* --- stepping without any allocation ------------------------------------------------------ */
/* The paper has no counterpart of this call; it serves callers that must not allocate device
 * memory while they run: real-time control loops that forbid allocation after start-up
 * (cudaMalloc and cudaFree can block on the device for an unbounded time), and frameworks that
 * hand out all device memory from their own pool and account for every byte.  They allocate the
 * arrays below once, their own way, and npx_step_noalloc steps them without allocating anything
 * (no cudaMalloc, cudaFree or allocating library routine is called).  Its scratch memory (work-
 * queue counter, step counter, scene schedule) is a static device array of the library that every
 * GPU which loads the library keeps until the process exits; its size limits a call to
 * NPX_NOALLOC_MAX_SCENES scenes (larger worlds are rejected with NPX_ERANGE).  All calls share
 * that array: calls whose work overlaps on the GPU (on different streams, or from different
 * threads) race on it and must be serialised by the caller.  The first call on a device looks up
 * the array's device address (a one-time set-up per device, done with that device current);
 * make that first call before capturing a stream.
 *
 * All pointers are DEVICE pointers to arrays the caller owns, in the layout a finalized world
 * uses internally (scene-major, points of each scene in ascending construction-frame height):
 *   link_off, point_off [S+1]; p0m [P*4] construction position xyz and mass; plink [P] link of
 *   each point; links [L] 48-byte records {anchor xyz, lo, unit axis xyz, hi (floats), parent,
 *   sensor bit, depth in the link tree, 0 (ints)}; gref [S*3] rest-pose CoG; mu [S]; hmap [S]
 *   (-1 flat); hm [maps*ny*nx] and hm_max [maps] (NULL when there are no maps); act / act_nu
 *   [J*4] / [J] actuator parameters and phase increments round(f dt 2^32);
 *   state [13*S] structure of arrays (component k of scene s at k*S+s: CoG xyz, quaternion
 *   wxyz, velocity xyz, angular momentum xyz); theta [J]; contact [P] flags of the last step;
 *   omega [S*3 as 3 rows of S]; sensors, status [S].
 * max_points and max_links must be at least the point and link counts of the largest scene (they
 * size the kernel's shared-memory slots; the call cannot check them without reading the device
 * arrays), and every hmap entry must be -1 or the index of one of the maps in hm.
 * step is the global step index of the first step (it fixes the joint-update phase and the
 * sinusoid phase).  The call reads it from this struct on the host when it is made; the caller
 * keeps the counter and advances it by n_steps between calls (the world is at step + n_steps
 * afterwards).  act_mode is NPX_ACT_HOLD or NPX_ACT_SINUSOID: machine-code controllers
 * (NPX_ACT_GP) need per-scene program state this struct does not carry and are refused with
 * NPX_EINVAL, as are height maps with hm_nx or hm_ny < 1 or hm_scale <= 0.  The call is
 * asynchronous on stream (a cudaStream_t, NULL = legacy default stream); state, theta, contact,
 * omega, sensors and status are read and written in place. */
#define NPX_NOALLOC_MAX_SCENES 65536
typedef struct {
    int n_scenes, max_points, max_links;
    const int *link_off, *point_off;
    const float *p0m;
    const uint8_t *plink;
    const void *links;
    const float *gref, *mu;
    const int *hmap;
    const float *hm, *hm_max;
    int hm_nx, hm_ny;
    float hm_scale, hm_origin[2];
    float dt, gravity[3];
    int joint_update_steps;
    float contact_omega, contact_zeta;
    int act_mode;
    const float *act;
    const uint32_t *act_nu;
    float *state, *theta;
    uint8_t *contact;
    float *omega;
    uint32_t *sensors, *status;
    int64_t step;
    int lanes_per_scene, warps_per_block;
} npx_device_world;
int npx_step_noalloc(const npx_device_world *world, int n_steps, void *stream);

#ifdef __cplusplus
}
#endif
#endif
