// npx_internal.h -- device data layout shared by the host library (npx_world.cpp) and the
// kernels (npx_step.cu).  Not part of the public C-ABI.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace npx {

// One link of a scene (48 bytes): hinge anchor and unit axis in the parent's construction frame
// (NeoPhysIx Appendix, createJoint), joint limits, parent link (scene-local, -1 for the root),
// contact-sensor bit (-1 none) and depth in the link tree (root 0).
struct LinkDev {
    float ax, ay, az, lo;
    float ux, uy, uz, hi;
    int parent, sensor, depth, pad;
};

// Dynamic state, structure of arrays: component k of scene s at st[k * S + s].
enum { ST_CX = 0, ST_CY, ST_CZ, ST_QW, ST_QX, ST_QY, ST_QZ, ST_VX, ST_VY, ST_VZ,
       ST_LX, ST_LY, ST_LZ, ST_N };

struct WorldDev {
    int S, P, L, J;
    const int *link_off, *point_off;      // [S+1]
    const float4 *p0m;                    // [P] construction position (xyz) and mass (w)
    const uint8_t *plink;                 // [P] scene-local link of each point
    const float *gref;                    // [3 * S] rest-pose CoG (centring reference of sums)
    const float *link_cog;                // [3 * L] CoG of each link's points, construction frame
    const LinkDev *links;                 // [L]
    const float *mu;                      // [S]
    const int *hmap;                      // [S] height map per scene, -1 = flat z = 0
    const float *hm;                      // [H * ny * nx]
    const float *hm_max;                  // [H] highest cell of each map
    int hm_nx, hm_ny;
    float hm_scale, hm_ox, hm_oy;
    float dt, gx, gy, gz;
    int K;
    float kw2, kc;                        // penalty: w_c^2 and 2 zeta w_c
    int act_mode;
    const float4 *act;                    // [J] amplitude, frequency, phase, bias
    const uint32_t *act_nu;               // [J] phase increment, 2^-32 turns per step
    // dynamic state
    float *st;                            // [ST_N * S]
    float *theta;                         // [J]
    uint8_t *kappa;                       // [P] contact flag of the last step
    float *omega;                         // [3 * S] angular velocity (output)
    uint32_t *sensors, *status;           // [S]
    // schedule
    const int *order;                     // [S] scenes, most points first
    int n_sched;                          // entries of order to run
    const int *sched_count;               // device count overriding n_sched, or NULL
    int max_points, max_links;
    const long long *step;                // device step counter n
    unsigned int *queue;                  // work-queue counter (reset before each launch)
    // 1: the launch takes the previous-step contacts from a detection at the current state
    // instead of kappa (after surrogate steps, which move scenes without detecting contacts)
    int reseed;
    // friction-model options: bit 0 rows weighted by the normal forces, bit 1 the friction
    // impulse's torque about the horizontal axes (0: Eqs. 1-6 as written)
    int fric_mode;
    // machine-code controller (act_mode 2, Sec. IV Table I): programs [32 * S], program counter
    // and accumulator [S], joint targets in 5-degree steps [J]
    const uint8_t *gp_prog;
    uint8_t *gp_pc, *gp_acc;
    int8_t *gp_k;
    // arenas: robots per arena (consecutive entries of the schedule, one warp; <= 1 = none) and
    // the radius of the sphere around every mass point for robot-robot contact
    int arena;
    float rc;
    // robot-robot broad phase: chunks of at most 16 points of one link (at most 64 per scene)
    const float4 *cbox;                   // [2 C] each chunk's construction-frame box: centre, half extent
    const int *cpo;                       // [C + 1] each chunk's entries in lpt
    const uint16_t *lpt;                  // [P] scene-local stored point indices, grouped by chunk
    const uint8_t *clink;                 // [C] scene-local link of each chunk
    const int *coff;                      // [S + 1] first chunk of each scene
    const uint8_t *pchunk;                // [P] scene-local chunk of each stored point
    int max_chunks;                       // chunks of the scene with the most
    // robot-robot pair lists (one per group of arenas a warp steps): point pairs of two robots of
    // an arena within reach plus a skin, alist_cap entries each, valid while the robots move less
    // than the skin between rebuilds
    uint32_t *alist;
    int alist_cap;
    // posed-shape cache (worlds stepped by the surrogate, whose plain launches are short): per
    // scene scache_mp + 2 scache_mt + 5 + 2 scache_ml float4 -- the posed offsets of its points,
    // the tile boxes of the lanes per scene that wrote them, the mass properties (4 float4),
    // (rmax, lanes per scene, 0, 0), and per link its orientation quaternion (w, x, y, z) and CoG
    // offset from the robot CoG (w = 0), both in the body frame.  Mode 0: unused; 1: written at
    // every shape update; 2: also read at launch entry instead of rebuilding the shape (every
    // scene's entry is current)
    float4 *scache;
    int scache_mp, scache_mt, scache_ml, scache_mode;
    // TMA map of the height maps [H][ny][nx] (FP32) in boxes of HM_BOX x HM_WIN x 1 cells for the
    // window loads, held on the host (hm_tmap_h) and passed to the step kernels as a parameter of
    // their own; hm_tma = 0 when the maps do not allow it (window loads by plain gathers)
    int hm_tma;
    const CUtensorMap *hm_tmap_h;
    // (height maps) the highest cell within hm_dr cells of every cell (a square, clamped to the
    // map) [H * ny * nx], or NULL: a scene's cull compares its tiles with the entry at its CoG's
    // cell while all its points stay within hm_dr cells of that cell, else with the map's highest
    const float *hm_dmax;
    int hm_dr;
};

struct LaunchCfg {
    int lps;      // lanes per scene: 4, 8, 16 or 32
    int wpb;      // warps per block
    int blocks;   // grid size
};

size_t step_smem_bytes(const WorldDev &W, int lps, int wpb);
int step_slot_bytes(const WorldDev &W, int lps);
int step_blocks_per_sm(const WorldDev &W, int lps, int wpb, cudaError_t *err);
cudaError_t launch_step(const WorldDev &W, const LaunchCfg &cfg, int n_steps, cudaStream_t st);
cudaError_t launch_advance(long long *d_step, int n, cudaStream_t st);
cudaError_t launch_init(const WorldDev &W, const float *d_origin, const float *d_quat,
                        const float *d_vel, const float *d_omega, cudaStream_t st);
cudaError_t launch_refresh(const WorldDev &W, cudaStream_t st);
// state exchange with the caller's layouts: AoS blocks <-> SoA state, contact flags between the
// caller's point order and the stored one (perm[i] = caller index of stored point i)
cudaError_t launch_scatter_state(const WorldDev &W, const float *aos, cudaStream_t st);
cudaError_t launch_gather_state(const WorldDev &W, float *aos, cudaStream_t st);
cudaError_t launch_permute_kappa(uint8_t *dst, const uint8_t *src, const int *perm, int P, bool to_stored,
                                 cudaStream_t st);
// ---- learned surrogate
// Per-scene posed shape (a function of the joint angles), rebuilt whenever they change.
struct SurCache {
    float4 *lk;       // [S * nl * 2]: per link, its orientation quaternion (w, x, y, z) in the body
                      //   frame, then its CoG offset from the robot CoG in the body frame (w = 0)
    float *inert;     // [12 * S]: body-frame inertia (xx yy zz xy xz yz), then its inverse
    float4 *spt;      // [S * nsp]: points of contact-sensor links, offset from the robot CoG in
                      //   the body frame; w = the sensor bit
    int *nsp_s;       // [S] sensor points of each scene
    int *sidx;        // [S * nsp]: their stored point index within the scene | sensor bit << 16
    int nsp, nl;      // capacity per scene; links per scene
};

struct SurrogateIO {
    int nf, nt, nl, ns;      // features, targets, links, sensor bits
    float *X;                // [S x nf] features (standardised when x_mu is set) or NULL
    void *Xb;                // [S x ldb] BF16 standardised features, zero-padded, or NULL
    int ldb;
    float *Xraw;             // [S x nf] raw features or NULL
    float *cxy_out;          // [S x 2] robot CoG (x, y) or NULL
    const float *cxy_ref;    // [S x 2] horizontal reference or NULL (the robot CoG)
    const float *prev;       // [S x nf] raw features of the previous state (delta target) or NULL
    float *T;                // [S x nt] delta target (standardised when t_mu is set) or NULL
    const float *x_mu, *x_isd, *t_mu, *t_sd;
};

cudaError_t launch_sensor_points(const WorldDev &W, int *count, int *max_count, cudaStream_t st);
// C.sidx: each scene's sensor points in stored order (once: the point-to-sensor map is static)
cudaError_t launch_sensor_index(const WorldDev &W, const SurCache &C, cudaStream_t st);
cudaError_t launch_shape_cache(const WorldDev &W, const SurCache &C, cudaStream_t st);
cudaError_t launch_features(const WorldDev &W, const SurCache &C, const SurrogateIO &io, cudaStream_t st);
// the surrogate's next state from the network output Y [S x ldy] (standardised deltas), kept
// where at most max_changed contact sensors change (with the sensors read at that state); the
// other scenes go to list / count, and their fallback counters fb [S] grow by one.  nx [16 * S],
// applied [S] and sens_new [S] are scratch.
cudaError_t launch_surrogate_update(const WorldDev &W, const SurCache &C, const float *Y, int ldy,
                                    const float *t_mu, const float *t_sd, float *nx, uint8_t *applied,
                                    uint32_t *sens_new, int *list, int *count, int *fb, int max_changed,
                                    cudaStream_t st);
cudaError_t launch_kappa_refresh(const WorldDev &W, const int *list, const int *count, cudaStream_t st);
// *total += *count * mult, then *count = 0
cudaError_t launch_accumulate(long long *total, int *count, int mult, cudaStream_t st);
// records msg as the thread's npx_last_error() text and returns code
int set_last_error(int code, const char *msg);
cudaError_t launch_points(const WorldDev &W, int scene, float *d_out, cudaStream_t st);
// Encodes *out for maps of at least 16 x 16 cells whose rows are a multiple of 16 bytes and sets
// W.hm_tma (1) and W.hm_tmap_h (out) on success; leaves hm_tma 0 otherwise (or when the encoder is
// unavailable).  out must outlive every launch of the world.
void encode_hm_tmap(WorldDev &W, int n_maps, CUtensorMap *out);
// out [H * ny * nx] = the highest cell of hm within R cells along x and y (clamped to the map);
// tmp is scratch of the same size
cudaError_t launch_hm_dilate(const float *hm, float *tmp, float *out, int H, int ny, int nx, int R,
                             cudaStream_t st);

}  // namespace npx

struct npx_mlp;
namespace npx {
// the surrogate network's stream, batch capacity and input / output widths
cudaStream_t mlp_stream(const npx_mlp *net);
int mlp_max_batch(const npx_mlp *net);
void mlp_dims(const npx_mlp *net, int *n_in, int *n_out);
// the network's packed BF16 input rows [max_batch x ld] (zero-padded columns), a forward pass of
// M rows from them, and the FP32 output rows [M x ld] it leaves (padded columns)
__nv_bfloat16 *mlp_input(npx_mlp *net, int *ld);
int mlp_forward_packed(npx_mlp *net, int M);
const float *mlp_output(const npx_mlp *net, int *ld);
}  // namespace npx
