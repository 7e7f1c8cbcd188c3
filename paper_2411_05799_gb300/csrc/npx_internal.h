// npx_internal.h -- device data layout shared by the host library (npx_world.cpp) and the
// kernels (npx_step.cu).  Not part of the public C-ABI.
#pragma once
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
};

struct LaunchCfg {
    int lps;      // lanes per scene: 8, 16 or 32
    int wpb;      // warps per block
    int blocks;   // grid size
};

size_t step_smem_bytes(const WorldDev &W, int lps, int wpb);
int step_blocks_per_sm(const WorldDev &W, int lps, int wpb, cudaError_t *err);
cudaError_t launch_step(const WorldDev &W, const LaunchCfg &cfg, int n_steps, cudaStream_t st);
cudaError_t launch_advance(long long *d_step, int n, cudaStream_t st);
cudaError_t launch_init(const WorldDev &W, const float *d_origin, const float *d_quat,
                        const float *d_vel, const float *d_omega, cudaStream_t st);
cudaError_t launch_refresh(const WorldDev &W, cudaStream_t st);
cudaError_t launch_features(const WorldDev &W, int nf, int nt, int nl, int ns, float *X, float *Xraw,
                            float *cxy_out, const float *cxy_ref, const float *prev, float *T,
                            const float *x_mu, const float *x_isd, const float *t_mu,
                            const float *t_sd, cudaStream_t st);
cudaError_t launch_surrogate_apply(const WorldDev &W, const float *Y, const float *t_mu,
                                   const float *t_sd, const float *F0, int nf, int nt,
                                   const float *cxy0, cudaStream_t st);
cudaError_t launch_contact_probe(const WorldDev &W, int *list, int *count, cudaStream_t st);
cudaError_t launch_restore(const WorldDev &W, const int *list, const int *count, const float *st_b,
                           const float *theta_b, const uint8_t *kappa_b, const uint32_t *sens_b,
                           const uint32_t *status_b, cudaStream_t st);
cudaError_t launch_accumulate(long long *total, int *count, cudaStream_t st);
// records msg as the thread's npx_last_error() text and returns code
int set_last_error(int code, const char *msg);
cudaError_t launch_points(const WorldDev &W, int scene, float *d_out, cudaStream_t st);

}  // namespace npx

struct npx_mlp;
namespace npx {
// the surrogate network's stream, batch capacity and input / output widths
cudaStream_t mlp_stream(const npx_mlp *net);
int mlp_max_batch(const npx_mlp *net);
void mlp_dims(const npx_mlp *net, int *n_in, int *n_out);
}  // namespace npx
