// npx_noalloc.cu -- npx_step_noalloc: the scene-step kernel on caller-owned device buffers, with
// its scratch memory in a fixed static device array instead of memory the library allocates.
//
// Who needs this: code that must not allocate device memory while it runs -- for example a
// real-time controller that forbids allocation after start-up (cudaMalloc and cudaFree can block
// on the device and take unbounded time), or a framework that hands out all device memory from
// its own pool and counts every byte.  Such callers allocate their arrays once, their own way,
// and pass them in; this entry point then adds no allocation of its own.
//
// The step kernel needs a little scratch besides its inputs and outputs: the counter of its
// persistent work queue, the global step counter it reads, and the schedule of scenes for the
// queue.  Here they live in g_noalloc_scratch, a file-scope device array that every GPU which
// loads the library holds until the process exits.  Its size fixes the largest world this entry
// point accepts: NOALLOC_MAX_SCENES scenes.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <string>

#include "../../include/npx.h"
#include "npx_internal.h"

namespace {

constexpr int NOALLOC_MAX_SCENES = 65536;
constexpr int NOALLOC_MAX_DEVICES = 64;
// layout: [0] work-queue counter (u32) | [2, 3] step counter (i64) | [4 ..) schedule (i32)
constexpr int NOALLOC_HEADER_WORDS = 4;

static __device__ __align__(256) unsigned int g_noalloc_scratch[NOALLOC_HEADER_WORDS + NOALLOC_MAX_SCENES];

// device address of g_noalloc_scratch per device, looked up once with that device current
unsigned int *g_scratch_ptr[NOALLOC_MAX_DEVICES] = {nullptr};

int noalloc_fail(int code, const char *msg) { return npx::set_last_error(code, msg); }

// Queue counter to zero, step counter to the caller's value, schedule = scenes in index order.
__global__ void noalloc_prepare(unsigned int *scratch, long long step, int n_scenes) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        scratch[0] = 0u;
        scratch[1] = 0u;
        *reinterpret_cast<long long *>(scratch + 2) = step;
    }
    if (i < n_scenes) scratch[NOALLOC_HEADER_WORDS + i] = (unsigned int)i;
}

}  // namespace

extern "C" int npx_step_noalloc(const npx_device_world *d, int n_steps, void *stream) {
    if (!d) return noalloc_fail(NPX_EINVAL, "npx_step_noalloc: null argument");
    if (n_steps < 0) return noalloc_fail(NPX_EINVAL, "npx_step_noalloc: n_steps must be >= 0");
    if (d->n_scenes < 1 || d->n_scenes > NOALLOC_MAX_SCENES) {
        char buf[160];
        snprintf(buf, sizeof buf, "npx_step_noalloc: %d scenes; this entry point takes 1 to %d scenes "
                 "(the size of its static scratch array)", d->n_scenes, NOALLOC_MAX_SCENES);
        return noalloc_fail(NPX_ERANGE, buf);
    }
    const int lps = d->lanes_per_scene, wpb = d->warps_per_block;
    if (lps != 4 && lps != 8 && lps != 16 && lps != 32)
        return noalloc_fail(NPX_EINVAL, "npx_step_noalloc: lanes_per_scene must be 4, 8, 16 or 32");
    if (wpb < 1 || wpb > 16) return noalloc_fail(NPX_EINVAL, "npx_step_noalloc: warps_per_block must be 1..16");
    if (d->max_points < 1 || d->max_points > 64 * lps || d->max_points > NPX_MAX_POINTS)
        return noalloc_fail(NPX_ERANGE, "npx_step_noalloc: max_points must be 1..64 * lanes_per_scene");
    if (d->max_links < 1 || d->max_links > NPX_MAX_LINKS) return noalloc_fail(NPX_ERANGE, "npx_step_noalloc: max_links out of range");
    // the machine-code controller needs per-scene program state this call has no fields for
    if (d->act_mode != NPX_ACT_HOLD && d->act_mode != NPX_ACT_SINUSOID)
        return noalloc_fail(NPX_EINVAL, "npx_step_noalloc: act_mode must be NPX_ACT_HOLD or NPX_ACT_SINUSOID "
                            "(the machine-code controller is not supported here)");
    if (!d->link_off || !d->point_off || !d->p0m || !d->plink || !d->links || !d->gref || !d->mu ||
        !d->hmap || !d->state || !d->theta || !d->contact || !d->omega || !d->sensors || !d->status ||
        (d->act_mode != NPX_ACT_HOLD && (!d->act || !d->act_nu)) ||
        (d->hm && !d->hm_max))
        return noalloc_fail(NPX_EINVAL, "npx_step_noalloc: null device array");
    // a map lookup clamps its cell index to [0, n - 1]: empty maps or a non-positive scale would
    // index outside the caller's array
    if (d->hm && (d->hm_nx < 1 || d->hm_ny < 1 || !(d->hm_scale > 0.f) || !std::isfinite(d->hm_scale) ||
                  !std::isfinite(d->hm_origin[0]) || !std::isfinite(d->hm_origin[1])))
        return noalloc_fail(NPX_EINVAL, "npx_step_noalloc: height maps need hm_nx >= 1, hm_ny >= 1, a finite "
                            "hm_scale > 0 and a finite origin");
    if (!(d->dt > 0.f) || d->joint_update_steps < 1 || d->step < 0)
        return noalloc_fail(NPX_EINVAL, "npx_step_noalloc: dt must be > 0, K >= 1, step >= 0");
    if (n_steps == 0) return NPX_OK;

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES)
        return noalloc_fail(NPX_ECUDA, "npx_step_noalloc: no usable current device");
    // set-up, once per device with that device current: the first call on a device looks up
    // the device address of the static scratch array
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            std::string m = std::string("npx_step_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e);
            return noalloc_fail(NPX_ECUDA, m.c_str());
        }
        g_scratch_ptr[dev] = static_cast<unsigned int *>(p);
    }
    unsigned int *scratch = g_scratch_ptr[dev];
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    // (W{} leaves hm_tma 0: the descriptor carries no map count to bound a TMA map, so height-map
    // windows load by plain gathers here)
    npx::WorldDev W{};
    W.S = d->n_scenes;
    W.link_off = d->link_off; W.point_off = d->point_off;
    W.p0m = reinterpret_cast<const float4 *>(d->p0m);
    W.plink = d->plink;
    W.gref = d->gref;
    W.links = static_cast<const npx::LinkDev *>(d->links);
    W.mu = d->mu; W.hmap = d->hmap;
    W.hm = d->hm; W.hm_max = d->hm_max;
    W.hm_nx = d->hm_nx; W.hm_ny = d->hm_ny; W.hm_scale = d->hm_scale;
    W.hm_ox = d->hm_origin[0]; W.hm_oy = d->hm_origin[1];
    W.dt = d->dt; W.gx = d->gravity[0]; W.gy = d->gravity[1]; W.gz = d->gravity[2];
    W.K = d->joint_update_steps;
    W.kw2 = d->contact_omega * d->contact_omega;
    W.kc = 2.f * d->contact_zeta * d->contact_omega;
    W.act_mode = d->act_mode;
    W.act = reinterpret_cast<const float4 *>(d->act);
    W.act_nu = d->act_nu;
    W.st = d->state; W.theta = d->theta; W.kappa = d->contact; W.omega = d->omega;
    W.sensors = d->sensors; W.status = d->status;
    W.max_points = d->max_points; W.max_links = d->max_links;
    W.queue = scratch;
    W.step = reinterpret_cast<const long long *>(scratch + 2);
    W.order = reinterpret_cast<const int *>(scratch + NOALLOC_HEADER_WORDS);
    W.n_sched = W.S;

    int nb = npx::step_blocks_per_sm(W, lps, wpb, &e);   // also raises the kernel's smem limit
    if (e != cudaSuccess || nb < 1)
        return noalloc_fail(NPX_ERANGE, "npx_step_noalloc: this launch shape does not fit on an SM");
    int n_sm = 0;
    if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return noalloc_fail(NPX_ECUDA, "npx_step_noalloc: device query failed");
    const int per_block = wpb * (32 / lps);
    int blocks = nb * n_sm;
    blocks = blocks < (W.S + per_block - 1) / per_block ? blocks : (W.S + per_block - 1) / per_block;
    noalloc_prepare<<<(W.S + 255) / 256, 256, 0, st>>>(scratch, (long long)d->step, W.S);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = npx::launch_step(W, {lps, wpb, blocks}, n_steps, st);
    if (e != cudaSuccess) {
        std::string m = std::string("npx_step_noalloc: launch failed: ") + cudaGetErrorString(e);
        return noalloc_fail(NPX_ECUDA, m.c_str());
    }
    return NPX_OK;
}
