// npx_step.cu -- the fused NeoPhysIx scene-step kernel for GB300 (sm_103a) and its helpers.
//
// Execution model.  A group of LPS lanes (4, 8, 16 or 32) of one warp owns one scene; a warp owns
// 32/LPS scenes.  Warps are persistent: each takes the next group of scenes from a global work
// counter (scenes ordered by decreasing point count), runs them through all n steps of the
// launch with their state in registers, writes them back and takes the next group.  Every
// reduction is a warp-synchronous xor-butterfly restricted to the group, so a scene never waits
// on a block-wide barrier and every lane of a group ends with bit-identical sums (and therefore
// bit-identical replicated scene state).
//
// Per scene the lanes hold, in shared memory, the point offsets r_i from the CoG in the shape
// frame together with the point masses (float4 per point), the link frames of the forward
// kinematics and the joint angles.  Contact history (one bit per point) lives in a 64-bit
// register per lane: point i belongs to lane i % LPS, bit i / LPS.
//
// The step (NeoPhysIx Sec. III; the readings of the paper that fix what it leaves open are the
// same as the CPU oracle's):
//   joint update (Sec. III-B, every K steps): clamped sinusoid targets, forward kinematics along
//     the link tree, new CoG and inertia; world CoG, root orientation and angular momentum kept;
//   collision (Sec. III-A): every point reads the ground height under it (flat, or a height map
//     indexed by floor((x - ox) * scale)); penalty force m (w_c^2 d - 2 zeta w_c vz) >= 0;
//   semi-implicit Euler of the CoG velocity and world angular momentum, exponential map of the
//     orientation;
//   friction (Sec. III-C, Eqs. 1-6): least squares over the points in contact in both steps,
//     solved in centred form (identical to the paper's 3x3 normal equations), a3 applied as a
//     rotation by asin(a3) about the contact centroid, dynamic part capped by mu * FN * dt.
#include <algorithm>
#include <cstring>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/npx.h"
#include "npx_internal.h"

namespace npx {

#define FULL_MASK 0xffffffffu

constexpr float POINT_RADIUS = 1e-3f;   // m, see shape_update
constexpr float CULL_MARGIN = 4e-3f;    // m, height margin of the candidate tiles (run_scene)
// height-map window kept in shared memory per scene (run_scene): HM_WIN x HM_WIN cells around the
// CoG (clamped to the map), moved when its centred origin drifts more than HM_DRIFT cells
constexpr int HM_WIN = 16, HM_DRIFT = 2;
// The window is stored as HM_WIN rows of HM_BOX cells: a TMA box starts on a 16-byte boundary, so
// its first column is the window's rounded down to a multiple of 4 and the window starts wsh
// (0..3) cells into each row; an mbarrier follows the window (HM_AREA bytes in all).
constexpr int HM_BOX = 20, HM_AREA = 1408;
constexpr unsigned long long HM_WAIT_NS = 1000000000ull;   // 1 s bound on a window load

// ------------------------------------------------------------------------ group reductions

template <int LPS, int N>
__device__ __forceinline__ void gsum(float (&v)[N]) {
#pragma unroll
    for (int o = LPS / 2; o > 0; o >>= 1) {
#pragma unroll
        for (int i = 0; i < N; ++i) v[i] += __shfl_xor_sync(FULL_MASK, v[i], o);
    }
}

template <int LPS>
__device__ __forceinline__ uint32_t gor(uint32_t v) {
#pragma unroll
    for (int o = LPS / 2; o > 0; o >>= 1) v |= __shfl_xor_sync(FULL_MASK, v, o);
    return v;
}

// ------------------------------------------------------------------------ small linear algebra

struct Sym {  // symmetric 3x3
    float xx, yy, zz, xy, xz, yz;
};

__device__ __forceinline__ void sym_mul(const Sym &a, const float x[3], float y[3]) {
    y[0] = a.xx * x[0] + a.xy * x[1] + a.xz * x[2];
    y[1] = a.xy * x[0] + a.yy * x[1] + a.yz * x[2];
    y[2] = a.xz * x[0] + a.yz * x[1] + a.zz * x[2];
}

__device__ __forceinline__ Sym sym_inv(const Sym &a) {
    float c00 = a.yy * a.zz - a.yz * a.yz;
    float c01 = a.xz * a.yz - a.xy * a.zz;
    float c02 = a.xy * a.yz - a.xz * a.yy;
    float det = a.xx * c00 + a.xy * c01 + a.xz * c02;
    float id = 1.0f / det;
    Sym r;
    r.xx = c00 * id;
    r.xy = c01 * id;
    r.xz = c02 * id;
    r.yy = (a.xx * a.zz - a.xz * a.xz) * id;
    r.yz = (a.xy * a.xz - a.xx * a.yz) * id;
    r.zz = (a.xx * a.yy - a.xy * a.xy) * id;
    return r;
}

// rotation matrix (row-major) of the unit quaternion (w, x, y, z)
__device__ __forceinline__ void quat_mat(const float q[4], float R[9]) {
    float w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z); R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z); R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y); R[7] = 2.f * (y * z + w * x); R[8] = 1.f - 2.f * (x * x + y * y);
}

__device__ __forceinline__ void mat_vec(const float R[9], const float x[3], float y[3]) {
    y[0] = R[0] * x[0] + R[1] * x[1] + R[2] * x[2];
    y[1] = R[3] * x[0] + R[4] * x[1] + R[5] * x[2];
    y[2] = R[6] * x[0] + R[7] * x[1] + R[8] * x[2];
}

__device__ __forceinline__ void mat_tvec(const float R[9], const float x[3], float y[3]) {
    y[0] = R[0] * x[0] + R[3] * x[1] + R[6] * x[2];
    y[1] = R[1] * x[0] + R[4] * x[1] + R[7] * x[2];
    y[2] = R[2] * x[0] + R[5] * x[1] + R[8] * x[2];
}

// world-frame tensor applied to x: R S R^T x
__device__ __forceinline__ void world_sym(const float R[9], const Sym &S, const float x[3], float y[3]) {
    float a[3], b[3];
    mat_tvec(R, x, a);
    sym_mul(S, a, b);
    mat_vec(R, b, y);
}

__device__ __forceinline__ void quat_mul(const float a[4], const float b[4], float c[4]) {
    float t0 = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    float t1 = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    float t2 = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    float t3 = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
    c[0] = t0; c[1] = t1; c[2] = t2; c[3] = t3;
}

// Small-angle sine/cosine and arcsine.  Inside |x| <= 1/16 the Taylor polynomials below are
// exact to single precision (first omitted terms x^7/5040, x^8/40320 and 35 x^9/1152 are below
// 1e-12); outside it the library functions are used.  Per-step rotation increments and friction
// corrections are almost always tiny, so this removes the range reduction from the hot path.
// (returned by value: a pointer into the caller would force its results into local memory)
__device__ __noinline__ float2 sincos_large(float x) {
    float s, c;
    sincosf(x, &s, &c);
    return make_float2(s, c);
}
__device__ __noinline__ float asin_large(float x) { return asinf(x); }

__device__ __forceinline__ void sincos_small(float x, float *s, float *c) {
    if (fabsf(x) <= 0.0625f) {
        const float x2 = x * x;
        *s = x * fmaf(x2, fmaf(x2, 1.f / 120.f, -1.f / 6.f), 1.f);
        *c = fmaf(x2, fmaf(x2, fmaf(x2, -1.f / 720.f, 1.f / 24.f), -0.5f), 1.f);
    } else {
        const float2 sc = sincos_large(x);
        *s = sc.x;
        *c = sc.y;
    }
}

__device__ __forceinline__ float asin_small(float x) {
    if (fabsf(x) <= 0.0625f) {
        const float x2 = x * x;
        return x * fmaf(x2, fmaf(x2, fmaf(x2, 5.f / 112.f, 3.f / 40.f), 1.f / 6.f), 1.f);
    }
    return asin_large(x);
}

// ------------------------------------------------------------------------ shared-memory slots

// Per scene: float4 pts[max_points] | float frames[12 * max_links] | float theta[max_links] |
// float theta_old[max_links] | float4 tile bounds[2 * ceil(max_points / lps)]
__host__ __device__ inline int tiles_offset(int max_points, int max_links) {
    return (16 * max_points + 56 * max_links + 15) & ~15;
}
__host__ __device__ inline int slot_bytes(int max_points, int max_links, int lps) {
    return tiles_offset(max_points, max_links) + 32 * ((max_points + lps - 1) / lps);
}
// (height maps) the window and its mbarrier after the slot, 128-byte aligned for the TMA box
__host__ __device__ inline int hm_win_offset(int max_points, int max_links, int lps) {
    return (slot_bytes(max_points, max_links, lps) + 127) & ~127;
}

// Bounding boxes for skipping points that cannot touch the ground.  Tile t holds points
// [t*LPS, (t+1)*LPS) of a scene (stored in ascending construction-frame height, so that a tile
// gathers points of similar height); tb[2t], tb[2t+1] are the min / max corners of the offsets r
// of its points, and c_z + min over that box of (R r)_z bounds their heights from below.
template <int LPS>
__device__ __noinline__ float tile_bounds(const float4 *pts, int np, float4 *tb, int gl) {
    __syncwarp();
    const int nt = (np + LPS - 1) / LPS;
    float r2 = 0.f;
    for (int t = gl; t < nt; t += LPS) {
        float4 lo = make_float4(INFINITY, INFINITY, INFINITY, 0.f);
        float4 hi = make_float4(-INFINITY, -INFINITY, -INFINITY, 0.f);
        const int b = t * LPS, n = min(np, b + LPS) - b;
#pragma unroll 4
        for (int j = 0; j < n; ++j) {
            // in full tiles each lane starts at a different point, so the group's loads hit
            // distinct banks
            const float4 r = pts[b + (n == LPS ? ((j + gl) & (LPS - 1)) : j)];
            lo.x = fminf(lo.x, r.x); lo.y = fminf(lo.y, r.y); lo.z = fminf(lo.z, r.z);
            hi.x = fmaxf(hi.x, r.x); hi.y = fmaxf(hi.y, r.y); hi.z = fmaxf(hi.z, r.z);
            r2 = fmaxf(r2, r.x * r.x + r.y * r.y + r.z * r.z);
        }
        tb[2 * t] = lo;
        tb[2 * t + 1] = hi;
    }
#pragma unroll
    for (int o = LPS / 2; o > 0; o >>= 1) r2 = fmaxf(r2, __shfl_xor_sync(FULL_MASK, r2, o));
    __syncwarp();
    return sqrtf(r2);   // the largest |r| of the scene's points (a bound for the cull margin)
}

// Body-frame box of a scene's posed points (the union of its tile boxes) as centre and half
// extent, the same on every lane of the group; a scene without points gets an empty box at 0.
template <int LPS>
__device__ __forceinline__ void robot_box(const float4 *tb, int ntiles, int gl, float (&bc)[3], float (&bh)[3]) {
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int t = gl; t < ntiles; t += LPS) {
        const float4 a = tb[2 * t], b = tb[2 * t + 1];
        lo[0] = fminf(lo[0], a.x); lo[1] = fminf(lo[1], a.y); lo[2] = fminf(lo[2], a.z);
        hi[0] = fmaxf(hi[0], b.x); hi[1] = fmaxf(hi[1], b.y); hi[2] = fmaxf(hi[2], b.z);
    }
#pragma unroll
    for (int o = LPS / 2; o > 0; o >>= 1) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            lo[i] = fminf(lo[i], __shfl_xor_sync(FULL_MASK, lo[i], o));
            hi[i] = fmaxf(hi[i], __shfl_xor_sync(FULL_MASK, hi[i], o));
        }
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const bool e = !(lo[i] <= hi[i]);
        bc[i] = e ? 0.f : 0.5f * (lo[i] + hi[i]);
        bh[i] = e ? 0.f : 0.5f * (hi[i] - lo[i]);
    }
}

// Tiles that may hold a point at or below the highest ground hmax: every lane tests the boxes of
// its tiles (t = gl, gl + LPS, ...) and ballots gather the group's answers into a mask.  The
// contact mask holds at most 64 tiles, so there are at most 64 / LPS rounds: all box tests are
// issued first (independent shared-memory loads), then the ballots.
// zfar receives the lowest box bottom among the tiles left out (+inf if none), the same for every
// lane of the group.
template <int LPS>
__device__ __forceinline__ uint64_t tiles_near_ground(const float4 *tb, int ntiles, const float R[9], float cz,
                                                      float hmax, int gl, float &zfar) {
    constexpr int ROUNDS = 64 / LPS;
    const int g = (threadIdx.x & 31) / LPS;
    bool near[ROUNDS];
    zfar = INFINITY;
#pragma unroll
    for (int r = 0; r < ROUNDS; ++r) {
        const int t = r * LPS + gl;
        near[r] = false;
        if (t < ntiles) {
            const float4 lo = tb[2 * t], hi = tb[2 * t + 1];
            const float zb = cz + fminf(R[6] * lo.x, R[6] * hi.x) + fminf(R[7] * lo.y, R[7] * hi.y) +
                             fminf(R[8] * lo.z, R[8] * hi.z);
            near[r] = zb <= hmax;
            if (!near[r]) zfar = fminf(zfar, zb);
        }
    }
#pragma unroll
    for (int o = LPS / 2; o > 0; o >>= 1) zfar = fminf(zfar, __shfl_xor_sync(FULL_MASK, zfar, o));
    uint64_t mask = 0;
#pragma unroll
    for (int r = 0; r < ROUNDS; ++r) {
        const uint32_t bal = __ballot_sync(FULL_MASK, near[r]);
        const uint64_t mine = (bal >> (g * LPS)) & (LPS == 32 ? 0xffffffffu : ((1u << LPS) - 1u));
        mask |= mine << (r * LPS);
    }
    return mask;
}

// ------------------------------------------------------------------------ kinematics (Sec. III-B)

// Link frames (rotation Q row-major, translation T) taking construction coordinates of each link
// to the shape frame (root link fixed).  A link's frame is its parent's frame followed by the
// hinge rotation by theta about the unit axis through the anchor.  Lanes build the local hinge
// transforms in parallel, then compose them one tree level at a time.
template <int LPS>
__device__ __noinline__ void link_frames(const WorldDev &W, int l0, int nl, const float *th, float *fr, int gl) {
    for (int l = gl; l < nl; l += LPS) {
        float *F = fr + 12 * l;
        if (l == 0) {
            F[0] = 1.f; F[1] = 0.f; F[2] = 0.f; F[3] = 0.f; F[4] = 1.f; F[5] = 0.f;
            F[6] = 0.f; F[7] = 0.f; F[8] = 1.f; F[9] = 0.f; F[10] = 0.f; F[11] = 0.f;
            continue;
        }
        const LinkDev lk = W.links[l0 + l];
        float s, c;
        sincosf(th[l - 1], &s, &c);
        const float k = 1.f - c, ux = lk.ux, uy = lk.uy, uz = lk.uz;
        float Rj[9] = {c + k * ux * ux, k * ux * uy - s * uz, k * ux * uz + s * uy,
                       k * uy * ux + s * uz, c + k * uy * uy, k * uy * uz - s * ux,
                       k * uz * ux - s * uy, k * uz * uy + s * ux, c + k * uz * uz};
        const float a[3] = {lk.ax, lk.ay, lk.az};
        float Ra[3];
        mat_vec(Rj, a, Ra);
#pragma unroll
        for (int i = 0; i < 9; ++i) F[i] = Rj[i];
        F[9] = a[0] - Ra[0]; F[10] = a[1] - Ra[1]; F[11] = a[2] - Ra[2];
    }
    __syncwarp();
    // level d >= 2: F_l = F_parent o F_l (parents at level d-1 are final)
    for (int d = 2;; ++d) {
        bool any = false;
        for (int l = gl; l < nl; l += LPS) {
            const LinkDev lk = W.links[l0 + l];
            if (lk.depth != d) continue;
            any = true;
            const float *P = fr + 12 * lk.parent;
            float *F = fr + 12 * l;
            float Q[9], T[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
#pragma unroll
                for (int j = 0; j < 3; ++j)
                    Q[3 * i + j] = P[3 * i] * F[j] + P[3 * i + 1] * F[3 + j] + P[3 * i + 2] * F[6 + j];
                T[i] = P[3 * i] * F[9] + P[3 * i + 1] * F[10] + P[3 * i + 2] * F[11] + P[9 + i];
            }
#pragma unroll
            for (int i = 0; i < 9; ++i) F[i] = Q[i];
            F[9] = T[0]; F[10] = T[1]; F[11] = T[2];
        }
        __syncwarp();
        if (!__any_sync(FULL_MASK, any)) break;
    }
}

// 16-byte asynchronous copy global -> shared (cp.async, completes at cp_async_wait_all)
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem_dst)),
                 "l"(gmem_src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ void fk_point(const float *fr, float4 a, int l, float p[3]) {
    const float *F = fr + 12 * l;
    p[0] = F[0] * a.x + F[1] * a.y + F[2] * a.z + F[9];
    p[1] = F[3] * a.x + F[4] * a.y + F[5] * a.z + F[10];
    p[2] = F[6] * a.x + F[7] * a.y + F[8] * a.z + F[11];
}

struct Shape {
    float M, g[3];
    Sym Ib, Ii;
};

// Posed shape as a pure function of the joint angles (Sec. III-A: the mass points give the CoG
// and the momentum; Sec. III-B: the segments move rigidly with their joints): link frames, one
// forward-kinematics pass that stores each point relative to the scene's rest CoG gref and sums
// the mass moments about it, then the CoG, the inertia about the CoG (parallel-axis theorem; gref
// is close to the CoG, so the FP32 sums do not cancel) and a recentring of the stored offsets.
// Being a function of theta alone, the result does not depend on where a launch (chunk) starts.
template <int LPS>
__device__ __noinline__ void shape_update(const WorldDev &W, int s, int p0, int np, int l0, int nl,
                                          const float *th, float *fr, float4 *pts, int gl,
                                          Shape &sh) {
    // the construction positions and masses go straight into the offsets array (asynchronous
    // copies, all in flight at once) and the points' links into the tile-box area (rebuilt after
    // every shape update) while the link frames are built
    uint8_t *lk = reinterpret_cast<uint8_t *>(pts) + tiles_offset(W.max_points, W.max_links);
#pragma unroll 8
    for (int i = gl; i < np; i += LPS) cp_async16(pts + i, W.p0m + p0 + i);
    {
        // the link bytes as whole aligned words (a quarter of the loads), the unaligned head and
        // tail byte by byte; every read stays inside the scene's bytes
        const uint8_t *src = W.plink + p0;
        const int h = min((int)((4u - ((uint32_t)(uintptr_t)src & 3u)) & 3u), np);
        const int nw = (np - h) >> 2;
        const uint32_t *ws = reinterpret_cast<const uint32_t *>(src + h);
        for (int i = gl; i < h; i += LPS) lk[i] = src[i];
#pragma unroll 4
        for (int k = gl; k < nw; k += LPS) {
            const uint32_t v = ws[k];
            uint8_t *d = lk + h + 4 * k;
            d[0] = (uint8_t)v; d[1] = (uint8_t)(v >> 8); d[2] = (uint8_t)(v >> 16); d[3] = (uint8_t)(v >> 24);
        }
        for (int i = h + 4 * nw + gl; i < np; i += LPS) lk[i] = src[i];
    }
    link_frames<LPS>(W, l0, nl, th, fr, gl);
    cp_async_wait_all();
    __syncwarp();
    const float gref[3] = {W.gref[3 * s], W.gref[3 * s + 1], W.gref[3 * s + 2]};
    float a[10] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
    for (int i = gl; i < np; i += LPS) {
        const float4 q = pts[i];
        float p[3];
        fk_point(fr, q, lk[i], p);
        const float dx = p[0] - gref[0], dy = p[1] - gref[1], dz = p[2] - gref[2], m = q.w;
        pts[i] = make_float4(dx, dy, dz, m);
        a[0] += m;
        a[1] += m * dx; a[2] += m * dy; a[3] += m * dz;
        a[4] += m * dx * dx; a[5] += m * dy * dy; a[6] += m * dz * dz;
        a[7] += m * dx * dy; a[8] += m * dx * dz; a[9] += m * dy * dz;
    }
    gsum<LPS, 10>(a);
    const float M = a[0], dx = a[1] / M, dy = a[2] / M, dz = a[3] / M;
    sh.M = M;
    sh.g[0] = gref[0] + dx; sh.g[1] = gref[1] + dy; sh.g[2] = gref[2] + dz;
    // inertia about the CoG = about gref minus the parallel-axis term; every mass point is also a
    // solid sphere of radius POINT_RADIUS (2/5 m r^2 about any axis), so that a single point or a
    // line of points still has an invertible inertia
    const float ps = 0.4f * M * POINT_RADIUS * POINT_RADIUS;
    sh.Ib.xx = (a[5] + a[6]) - M * (dy * dy + dz * dz) + ps;
    sh.Ib.yy = (a[4] + a[6]) - M * (dx * dx + dz * dz) + ps;
    sh.Ib.zz = (a[4] + a[5]) - M * (dx * dx + dy * dy) + ps;
    sh.Ib.xy = -a[7] + M * dx * dy;
    sh.Ib.xz = -a[8] + M * dx * dz;
    sh.Ib.yz = -a[9] + M * dy * dz;
    sh.Ii = sym_inv(sh.Ib);
    for (int i = gl; i < np; i += LPS) {
        float4 r = pts[i];
        r.x -= dx; r.y -= dy; r.z -= dz;
        pts[i] = r;
    }
    __syncwarp();
}

// unit quaternion of a rotation matrix (row-major), sign chosen with w >= 0
__device__ __forceinline__ void quat_from_mat(const float *Q, float *q) {
    const float tr = Q[0] + Q[4] + Q[8];
    float w, x, y, z;
    if (tr > 0.f) {
        const float s = 2.f * sqrtf(tr + 1.f);
        w = 0.25f * s; x = (Q[7] - Q[5]) / s; y = (Q[2] - Q[6]) / s; z = (Q[3] - Q[1]) / s;
    } else if (Q[0] > Q[4] && Q[0] > Q[8]) {
        const float s = 2.f * sqrtf(1.f + Q[0] - Q[4] - Q[8]);
        w = (Q[7] - Q[5]) / s; x = 0.25f * s; y = (Q[1] + Q[3]) / s; z = (Q[2] + Q[6]) / s;
    } else if (Q[4] > Q[8]) {
        const float s = 2.f * sqrtf(1.f + Q[4] - Q[0] - Q[8]);
        w = (Q[2] - Q[6]) / s; x = (Q[1] + Q[3]) / s; y = 0.25f * s; z = (Q[5] + Q[7]) / s;
    } else {
        const float s = 2.f * sqrtf(1.f + Q[8] - Q[0] - Q[4]);
        w = (Q[3] - Q[1]) / s; x = (Q[2] + Q[6]) / s; y = (Q[5] + Q[7]) / s; z = 0.25f * s;
    }
    const float sg = w < 0.f ? -1.f : 1.f;
    q[0] = sg * w; q[1] = sg * x; q[2] = sg * y; q[3] = sg * z;
}

// ------------------------------------------------------------------------ posed-shape cache

__host__ __device__ inline long long scache_stride(int mp, int mt, int ml) {
    return (long long)mp + 2 * mt + 5 + 2 * ml;
}

// Writes the scene's posed shape (pts, tile boxes, mass properties, and each link's orientation and
// CoG offset in the body frame from its frame in fr) to its cache entry; stores only.
template <int LPS>
__device__ __forceinline__ void scache_store(const WorldDev &W, int s, int np, const float4 *pts, const float4 *tb,
                                             const Shape &sh, float rmax, const float *fr, int l0, int nl, int gl) {
    float4 *e = W.scache + (size_t)s * scache_stride(W.scache_mp, W.scache_mt, W.scache_ml);
    const int nt = (np + LPS - 1) / LPS;
    for (int i = gl; i < np; i += LPS) e[i] = pts[i];
    for (int i = gl; i < 2 * nt; i += LPS) e[W.scache_mp + i] = tb[i];
    float4 *lk = e + W.scache_mp + 2 * W.scache_mt + 5;
    for (int l = gl; l < nl; l += LPS) {
        const float *F = fr + 12 * l;
        const float pc0 = W.link_cog[3 * (l0 + l)], pc1 = W.link_cog[3 * (l0 + l) + 1], pc2 = W.link_cog[3 * (l0 + l) + 2];
        float ql[4];
        quat_from_mat(F, ql);
        lk[2 * l] = make_float4(ql[0], ql[1], ql[2], ql[3]);
        lk[2 * l + 1] = make_float4(F[0] * pc0 + F[1] * pc1 + F[2] * pc2 + F[9] - sh.g[0],
                                    F[3] * pc0 + F[4] * pc1 + F[5] * pc2 + F[10] - sh.g[1],
                                    F[6] * pc0 + F[7] * pc1 + F[8] * pc2 + F[11] - sh.g[2], 0.f);
    }
    if (gl == 0) {
        float4 *m = e + W.scache_mp + 2 * W.scache_mt;
        m[0] = make_float4(sh.M, sh.g[0], sh.g[1], sh.g[2]);
        m[1] = make_float4(sh.Ib.xx, sh.Ib.yy, sh.Ib.zz, sh.Ib.xy);
        m[2] = make_float4(sh.Ib.xz, sh.Ib.yz, sh.Ii.xx, sh.Ii.yy);
        m[3] = make_float4(sh.Ii.zz, sh.Ii.xy, sh.Ii.xz, sh.Ii.yz);
        m[4] = make_float4(rmax, __int_as_float(LPS), 0.f, 0.f);
    }
}

// Reads the posed shape of scene s (-1: no scene) from its cache entry into the slot: the offsets,
// the mass properties and, when they were written with this many lanes per scene on every scene
// of the warp, the tile boxes (else they are rebuilt from the offsets).  Returns rmax.
template <int LPS>
__device__ __forceinline__ float scache_load(const WorldDev &W, int s, int np, float4 *pts, float4 *tb, Shape &sh,
                                             int gl) {
    const float4 *e = W.scache + (size_t)(s < 0 ? 0 : s) * scache_stride(W.scache_mp, W.scache_mt, W.scache_ml);
    const int nt = (np + LPS - 1) / LPS;
    const float4 *m = e + W.scache_mp + 2 * W.scache_mt;
    float4 m0 = make_float4(1.f, 0.f, 0.f, 0.f), m1 = make_float4(1.f, 1.f, 1.f, 0.f);
    float4 m2 = make_float4(0.f, 0.f, 1.f, 1.f), m3 = make_float4(1.f, 0.f, 0.f, 0.f);
    float4 m4 = make_float4(0.f, __int_as_float(LPS), 0.f, 0.f);
    if (s >= 0) { m0 = m[0]; m1 = m[1]; m2 = m[2]; m3 = m[3]; m4 = m[4]; }
    const bool tb_ok = __all_sync(FULL_MASK, __float_as_int(m4.y) == LPS);
#pragma unroll 4
    for (int i = gl; i < np; i += LPS) cp_async16(pts + i, e + i);
    if (tb_ok)
        for (int i = gl; i < 2 * nt; i += LPS) cp_async16(tb + i, e + W.scache_mp + i);
    cp_async_wait_all();
    __syncwarp();
    sh.M = m0.x; sh.g[0] = m0.y; sh.g[1] = m0.z; sh.g[2] = m0.w;
    sh.Ib = Sym{m1.x, m1.y, m1.z, m1.w, m2.x, m2.y};
    sh.Ii = Sym{m2.z, m2.w, m3.x, m3.y, m3.z, m3.w};
    if (tb_ok) return m4.x;
    return tile_bounds<LPS>(pts, np, tb, gl);   // every lane of the warp takes this branch
}

// ------------------------------------------------------------------------ ground (Sec. III-A)

template <bool FLAT>
__device__ __forceinline__ float ground(const WorldDev &W, int hm, float x, float y) {
    if (FLAT || hm < 0) return 0.f;
    const float fx = __fmul_rn(__fsub_rn(x, W.hm_ox), W.hm_scale);
    const float fy = __fmul_rn(__fsub_rn(y, W.hm_oy), W.hm_scale);
    int ix = __float2int_rd(fx), iy = __float2int_rd(fy);
    ix = min(max(ix, 0), W.hm_nx - 1);
    iy = min(max(iy, 0), W.hm_ny - 1);
    return __ldg(W.hm + ((size_t)hm * W.hm_ny + iy) * W.hm_nx + ix);
}

// The same lookup through a window of the scene's map in shared memory.  The window (origin
// wx0, wy0 >= 0) holds the height at the clamped index of each of its cells, so an unclamped index
// inside it already reads the clamped cell's height; others are clamped and read from global
// memory (the same value either way).
template <bool FLAT>
__device__ __forceinline__ float ground_win(const WorldDev &W, int hm, const float *win, int wx0, int wy0, float x,
                                            float y) {
    if (FLAT || hm < 0) return 0.f;
    const float fx = __fmul_rn(__fsub_rn(x, W.hm_ox), W.hm_scale);
    const float fy = __fmul_rn(__fsub_rn(y, W.hm_oy), W.hm_scale);
    int ix = __float2int_rd(fx), iy = __float2int_rd(fy);
    const unsigned ux = (unsigned)ix - (unsigned)wx0, uy = (unsigned)iy - (unsigned)wy0;
    if (ux < (unsigned)HM_WIN && uy < (unsigned)HM_WIN) return win[uy * HM_BOX + ux];
    ix = min(max(ix, 0), W.hm_nx - 1);
    iy = min(max(iy, 0), W.hm_ny - 1);
    return __ldg(W.hm + ((size_t)hm * W.hm_ny + iy) * W.hm_nx + ix);
}

// Window loads with TMA: one 3-D box (HM_BOX x HM_WIN cells of map hm) into shared memory,
// completing on the scene's mbarrier, waited for with a bound.
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void win_bar_init(uint64_t *b) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(b)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void win_bar_inval(uint64_t *b) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(b)) : "memory");
}
__device__ __forceinline__ void win_load(float *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *b) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)),
                 "r"((uint32_t)(HM_BOX * HM_WIN * sizeof(float)))
                 : "memory");
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_addr(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(b))
        : "memory");
}
// The whole warp waits for the window loads of its groups: lanes with `mine` set poll their
// group's barrier for phase `parity` (a non-blocking test); the loop ends for all lanes at once,
// when every lane is done or when HM_WAIT_NS have passed, so the groups leave it converged (a
// per-group wait loop left them diverged for the rest of the launch).  Returns, per lane, whether
// its load landed (true for lanes without one).  All 32 lanes must call it.
__device__ __forceinline__ bool win_wait_warp(uint64_t *b, uint32_t parity, bool mine) {
    bool done = !mine;
    unsigned long long t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (;;) {
        if (!done) {
            uint32_t ok;
            asm volatile(
                "{\n\t.reg .pred p;\n\t"
                "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                "selp.u32 %0, 1, 0, p;\n\t}"
                : "=r"(ok)
                : "r"(smem_addr(b)), "r"(parity)
                : "memory");
            done = ok != 0;
        }
        if (__all_sync(FULL_MASK, done)) return true;
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (__any_sync(FULL_MASK, t - t0 > HM_WAIT_NS)) return done;
    }
}

// ------------------------------------------------------------------------ actuators (Sec. III-B)

__device__ __forceinline__ float joint_target(const WorldDev &W, int j, long long n) {
    const float4 a = W.act[j];
    const uint32_t u = W.act_nu[j] * (uint32_t)(unsigned long long)n;   // phase mod 1 turn, exact
    const float turns = __uint2float_rn(u) * 2.3283064365386963e-10f;
    return a.w + a.x * sinf(fmaf(6.2831853071795865f, turns, a.z));
}

// ------------------------------------------------------------------------ machine-code controller

constexpr int GP_LEN = 32, GP_PER_UPDATE = 32, GP_KMAX = 36;
constexpr float GP_STEP = 0.087266462599716478846f;   // 5 degrees

// The controller of Sec. IV at a joint update, run by lane 0 of the scene's group: GP_PER_UPDATE
// instructions of Table I from the saved program counter.  8-bit opcode = 3-bit command + 5-bit
// value x: 000 / 001 move motor x left / right (its target by -/+ one 5-degree step, saturating at
// +-GP_KMAX; motors the scene lacks are ignored), 010 acc = foot-contact bit x of the last step,
// 011 acc = x, 100 jump to x if acc != 0, 101 acc = ~acc, 110 inc, 111 dec (8-bit accumulator,
// the program counter wraps after address 31).
__device__ __noinline__ void gp_run(const WorldDev &W, int s, int j0, int nj, uint32_t sensors) {
    const uint8_t *prog = W.gp_prog + (size_t)GP_LEN * s;
    int8_t *k = W.gp_k + j0;
    uint32_t p = W.gp_pc[s] & (GP_LEN - 1), a = W.gp_acc[s];
    for (int it = 0; it < GP_PER_UPDATE; ++it) {
        const uint32_t ins = prog[p], op = ins >> 5, x = ins & 31u;
        uint32_t next = (p + 1) & (GP_LEN - 1);
        switch (op) {
            case 0: if ((int)x < nj && k[x] > -GP_KMAX) k[x] = (int8_t)(k[x] - 1); break;
            case 1: if ((int)x < nj && k[x] < GP_KMAX) k[x] = (int8_t)(k[x] + 1); break;
            case 2: a = (sensors >> x) & 1u; break;
            case 3: a = x; break;
            case 4: if (a != 0u) next = x; break;
            case 5: a = ~a & 255u; break;
            case 6: a = (a + 1u) & 255u; break;
            default: a = (a + 255u) & 255u; break;
        }
        p = next;
    }
    W.gp_pc[s] = (uint8_t)p;
    W.gp_acc[s] = (uint8_t)a;
}

// ------------------------------------------------------------------------ robot-robot contact

// Arenas (robot-robot collision, the extension named as future work): the W.arena robots of an
// arena are consecutive groups of one warp.  Every mass point is a sphere of radius W.rc; two
// points of different robots closer than 2 rc push apart along the line through them with the
// ground contact's penalty law written for the pair (stiffness m_r w_c^2, damping 2 zeta m_r w_c,
// m_r the pair's reduced mass), no adhesion, no friction between robots.
//
// Broad phase by chunks: each link's points are cut along the link's longest axis into chunks of
// at most 16 points (at most 64 per robot; W.cbox, W.clink, W.cpo / W.lpt, W.pchunk).  At every
// shape update each robot turns its chunks' construction-frame boxes into body-frame boxes with
// the new link frames.  Each step, after the joint update, it publishes in its exchange area
// (after all slots of the block) its CoG, rotation, velocity, angular velocity, point and chunk
// ranges, the world box of all its points and the world boxes of its chunks.  Then the whole warp
// takes the robot pairs (i < j) of its arenas one at a time, so that its lanes follow one control
// flow: if the pair's world boxes come within 2 rc, the lanes mark for each chunk of i the chunks
// of j whose boxes come within 2 rc of it (a 64-bit mask in shared memory), then spread over i's
// points; a point of a marked chunk goes into j's body frame once, is tested against each marked
// chunk's body-frame box and then against that chunk's stored offsets.  Each pair force acts on
// both robots (F on i, -F on j); the warp sums the pair's wrenches and adds them to the two
// robots' totals in shared memory, pair after pair in a fixed order.  All culls are conservative
// (a margin covers the rounding of the boxes), so the forces are those of all pairs within reach.
constexpr float ARENA_MARGIN = 1e-4f;   // m, added to every cull distance
enum { XC_C = 0, XC_R = 3, XC_V = 12, XC_W = 15, XC_BC = 18, XC_BH = 21, XC_ACTIVE = 24, XC_C0 = 25,
       XC_NC = 26, XC_P0 = 27, XC_NP = 28, XC_RF = 32, XC_D = 38, XC_CREF = 39, XC_RREF = 42, XC_LH = 51,
       XC_N = 64 };
// Pair lists (Verlet lists): the point pairs of each robot pair of the warp's arenas closer than
// reach + skin (skin = 2 rc) at the last rebuild.  A point of robot i has since moved at most
// |c_i - c_i,ref| + ||R_i - R_i,ref||_2 r_max,i (the posed shape is rigid between joint updates);
// for rotations R - R_ref has two equal singular values, so ||.||_2 = ||.||_F / sqrt(2) (up to the
// rounding of the matrices, which a small allowance covers).  While these bounds of two robots sum
// to less than the skin, no pair left out can be within reach.  The lists are rebuilt at a launch's first step, at joint updates and when a bound
// runs out; entries are appended in a fixed order (ballots), so results are deterministic.  The
// list header (in the first robot's exchange area): state (0 none, 1 valid, 2 overflowed: the
// full pass serves until the next rebuild) and each pair's end offset.
constexpr int AL_BITS = 11;   // bits of a point index in an entry (at most 2,048 points a robot)

// Exchange area of a scene: XC_N floats of state and wrench totals | world chunk boxes
// [max_chunks] (2 float4) | body chunk boxes [max_chunks] (2 float4) | near masks [max_chunks]
// (uint64)
__host__ __device__ inline int xch_bytes(int max_chunks) { return (4 * XC_N + 72 * max_chunks + 15) & ~15; }

// body-frame boxes of the scene's chunks from the current frames of their links (centre Q c + T - g,
// half extent |Q| h; g the posed CoG in the shape frame)
template <int LPS>
__device__ __forceinline__ void chunk_boxes_body(const WorldDev &W, int c0, int nc, const float *fr, const float g[3],
                                                 float4 *LB, int gl) {
    for (int l = gl; l < nc; l += LPS) {
        const float4 cc = W.cbox[2 * (c0 + l)], hh = W.cbox[2 * (c0 + l) + 1];
        const float *F = fr + 12 * W.clink[c0 + l];
        float4 cb, hb;
        cb.x = F[0] * cc.x + F[1] * cc.y + F[2] * cc.z + F[9] - g[0];
        cb.y = F[3] * cc.x + F[4] * cc.y + F[5] * cc.z + F[10] - g[1];
        cb.z = F[6] * cc.x + F[7] * cc.y + F[8] * cc.z + F[11] - g[2];
        hb.x = fabsf(F[0]) * hh.x + fabsf(F[1]) * hh.y + fabsf(F[2]) * hh.z;
        hb.y = fabsf(F[3]) * hh.x + fabsf(F[4]) * hh.y + fabsf(F[5]) * hh.z;
        hb.z = fabsf(F[6]) * hh.x + fabsf(F[7]) * hh.y + fabsf(F[8]) * hh.z;
        cb.w = hb.w = 0.f;
        LB[2 * l] = cb;
        LB[2 * l + 1] = hb;
    }
    __syncwarp();
}

__device__ __forceinline__ bool boxes_meet(float4 ca, float4 ha, float4 cb, float4 hb, float cull) {
    return fabsf(ca.x - cb.x) <= ha.x + hb.x + cull && fabsf(ca.y - cb.y) <= ha.y + hb.y + cull &&
           fabsf(ca.z - cb.z) <= ha.z + hb.z + cull;
}

// The pair force of point a of robot i and point b of robot j closer than reach (d = a - b in j's
// body frame, dd = |d|^2 > 0; ra, and rb = Rj pb, their offsets from the robots' CoGs): F along
// the line of centres with the contact law, F on i and -F on j, added to both wrenches.
__device__ __forceinline__ void pair_force(float4 pa, float4 pb, const float ra[3], float d0, float d1, float d2,
                                           float dd, const float Rj[9], const float vi[3], const float wi[3],
                                           const float vj[3], const float wj[3], float reach, float kw2, float kc,
                                           float (&fi)[6], float (&fj)[6]) {
    const float dist = sqrtf(dd), inv = 1.f / dist;
    const float hn[3] = {d0 * inv, d1 * inv, d2 * inv};
    float n[3], rb[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        n[k] = Rj[3 * k] * hn[0] + Rj[3 * k + 1] * hn[1] + Rj[3 * k + 2] * hn[2];
        rb[k] = Rj[3 * k] * pb.x + Rj[3 * k + 1] * pb.y + Rj[3 * k + 2] * pb.z;
    }
    const float va[3] = {vi[0] + (wi[1] * ra[2] - wi[2] * ra[1]),
                         vi[1] + (wi[2] * ra[0] - wi[0] * ra[2]),
                         vi[2] + (wi[0] * ra[1] - wi[1] * ra[0])};
    const float vb[3] = {vj[0] + (wj[1] * rb[2] - wj[2] * rb[1]),
                         vj[1] + (wj[2] * rb[0] - wj[0] * rb[2]),
                         vj[2] + (wj[0] * rb[1] - wj[1] * rb[0])};
    const float vn = (va[0] - vb[0]) * n[0] + (va[1] - vb[1]) * n[1] + (va[2] - vb[2]) * n[2];
    const float mr = pa.w * pb.w / (pa.w + pb.w);
    const float f = fmaxf(0.f, mr * (kw2 * (reach - dist) - kc * vn));
    const float F[3] = {f * n[0], f * n[1], f * n[2]};
    fi[0] += F[0]; fi[1] += F[1]; fi[2] += F[2];
    fi[3] += ra[1] * F[2] - ra[2] * F[1];
    fi[4] += ra[2] * F[0] - ra[0] * F[2];
    fi[5] += ra[0] * F[1] - ra[1] * F[0];
    fj[0] -= F[0]; fj[1] -= F[1]; fj[2] -= F[2];
    fj[3] -= rb[1] * F[2] - rb[2] * F[1];
    fj[4] -= rb[2] * F[0] - rb[0] * F[2];
    fj[5] -= rb[0] * F[1] - rb[1] * F[0];
}

// The pair list of the warp's arenas from the exchange areas (see above): entries ia | ib << AL_BITS
// per robot pair, in pair order; returns the entries written (more than cap: overflowed).
__device__ __forceinline__ int arena_build(const WorldDev &W, unsigned char *xw, const unsigned char *pw, int sbytes,
                                           int XB, int G, float cut, uint32_t *alist) {
    const int lane = threadIdx.x & 31, A = W.arena, per_arena = A * (A - 1) / 2;
    // (the margin covers the rounding of the distances, so a pair left out was farther than cut)
    const float cull = cut + ARENA_MARGIN, cut2 = cull * cull;
    float *X0 = reinterpret_cast<float *>(xw);
    int total = 0;
    for (int pr = 0; pr < (G / A) * per_arena; ++pr) {   // the same pairs, in the same order, on every lane
        int i = 0, t = pr % per_arena;
        while (t >= A - 1 - i) { t -= A - 1 - i; ++i; }
        const int gi = (pr / per_arena) * A + i, gj = gi + 1 + t;
        const float *Xi = reinterpret_cast<const float *>(xw + gi * XB);
        const float *Xj = reinterpret_cast<const float *>(xw + gj * XB);
        bool ov = Xi[XC_ACTIVE] != 0.f && Xj[XC_ACTIVE] != 0.f;
#pragma unroll
        for (int k = 0; k < 3; ++k) ov = ov && fabsf(Xi[XC_BC + k] - Xj[XC_BC + k]) <= Xi[XC_BH + k] + Xj[XC_BH + k] + cull;
        if (ov) {   // read from shared memory: the same on every lane
            const float4 *LWi = reinterpret_cast<const float4 *>(xw + gi * XB + 4 * XC_N);
            const float4 *LWj = reinterpret_cast<const float4 *>(xw + gj * XB + 4 * XC_N);
            const float4 *LBj = LWj + 2 * W.max_chunks;
            uint64_t *NMi = reinterpret_cast<uint64_t *>(xw + gi * XB + 4 * XC_N + 64 * W.max_chunks);
            const int nli = __float_as_int(Xi[XC_NC]), nlj = __float_as_int(Xj[XC_NC]);
            const int p0i = __float_as_int(Xi[XC_P0]), npi = __float_as_int(Xi[XC_NP]);
            const int l0j = __float_as_int(Xj[XC_C0]);
            const float4 bcj = make_float4(Xj[XC_BC], Xj[XC_BC + 1], Xj[XC_BC + 2], 0.f);
            const float4 bhj = make_float4(Xj[XC_BH], Xj[XC_BH + 1], Xj[XC_BH + 2], 0.f);
            for (int l = lane; l < nli; l += 32) {
                uint64_t nm = 0;
                const float4 ca = LWi[2 * l], ha = LWi[2 * l + 1];
                if (boxes_meet(ca, ha, bcj, bhj, cull))
                    for (int lb = 0; lb < nlj; ++lb)
                        if (boxes_meet(ca, ha, LWj[2 * lb], LWj[2 * lb + 1], cull)) nm |= 1ull << lb;
                NMi[l] = nm;
            }
            __syncwarp();
            float ci[3], Ri[9], cj[3], Rj[9];
#pragma unroll
            for (int k = 0; k < 3; ++k) { ci[k] = Xi[XC_C + k]; cj[k] = Xj[XC_C + k]; }
#pragma unroll
            for (int k = 0; k < 9; ++k) { Ri[k] = Xi[XC_R + k]; Rj[k] = Xj[XC_R + k]; }
            const float4 *pti = reinterpret_cast<const float4 *>(pw + (ptrdiff_t)gi * sbytes);
            const float4 *ptj = reinterpret_cast<const float4 *>(pw + (ptrdiff_t)gj * sbytes);
            for (int ia0 = 0; ia0 < npi; ia0 += 32) {   // warp-uniform
                const int ia = ia0 + lane;
                uint64_t bm = ia < npi ? NMi[W.pchunk[p0i + ia]] : 0ull;
                float ah0 = 0.f, ah1 = 0.f, ah2 = 0.f;
                if (bm) {
                    const float4 pa = pti[ia];
                    float e[3];
#pragma unroll
                    for (int k = 0; k < 3; ++k)
                        e[k] = (ci[k] + (Ri[3 * k] * pa.x + Ri[3 * k + 1] * pa.y + Ri[3 * k + 2] * pa.z)) - cj[k];
                    ah0 = Rj[0] * e[0] + Rj[3] * e[1] + Rj[6] * e[2];
                    ah1 = Rj[1] * e[0] + Rj[4] * e[1] + Rj[7] * e[2];
                    ah2 = Rj[2] * e[0] + Rj[5] * e[1] + Rj[8] * e[2];
                }
                // each lane walks its candidate chunks: a round takes the lane's next chunk when
                // its current one is done (whose body-frame box must come within reach) and tests
                // up to 16 of the chunk's points at once; the rounds are warp-wide and the lanes'
                // entries go out in lane order (a warp prefix sum), so the appends keep a fixed
                // order
                int ib = 0, b1 = 0;
                while (__any_sync(FULL_MASK, bm != 0ull || ib < b1)) {
                    uint32_t hit = 0u;
                    int ib0 = 0;   // the round's first tested point
                    if (ib >= b1 && bm) {
                        const int lb = __ffsll((long long)bm) - 1;
                        bm &= bm - 1;
                        const float4 cbh = LBj[2 * lb], hbh = LBj[2 * lb + 1];
                        if (fabsf(ah0 - cbh.x) <= hbh.x + cull && fabsf(ah1 - cbh.y) <= hbh.y + cull &&
                            fabsf(ah2 - cbh.z) <= hbh.z + cull) {
                            ib = W.cpo[l0j + lb];
                            b1 = W.cpo[l0j + lb + 1];
                        }
                    }
                    if (ib < b1) {
                        ib0 = ib;
                        const int nb = min(16, b1 - ib);
#pragma unroll
                        for (int k = 0; k < 16; ++k) {
                            if (k < nb) {
                                const float4 pb = ptj[__ldg(W.lpt + ib + k)];
                                const float d0 = ah0 - pb.x, d1 = ah1 - pb.y, d2 = ah2 - pb.z;
                                if (d0 * d0 + d1 * d1 + d2 * d2 < cut2) hit |= 1u << k;
                            }
                        }
                        ib += nb;
                    }
                    const int cnt = __popc(hit);
                    int pre = cnt;   // inclusive prefix sum over the lanes
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int y = __shfl_up_sync(FULL_MASK, pre, o);
                        if (lane >= o) pre += y;
                    }
                    int pos = total + pre - cnt;
                    for (uint32_t h = hit; h; h &= h - 1, ++pos) {
                        const int k = __ffs(h) - 1;
                        if (pos < W.alist_cap)
                            alist[pos] = (uint32_t)ia | ((uint32_t)__ldg(W.lpt + ib0 + k) << AL_BITS);
                    }
                    total += __shfl_sync(FULL_MASK, pre, 31);
                }
            }
        }
        if (lane == 0) X0[XC_LH + 1 + pr] = __int_as_float(total);
        __syncwarp();
    }
    return total;
}

// Pair forces from the list: for each robot pair of the warp, its entries spread over the lanes,
// the pair's wrenches summed by the warp and added to the two robots' totals, pair after pair.
__device__ __forceinline__ void arena_list_forces(const WorldDev &W, unsigned char *xw, const unsigned char *pw,
                                                  int sbytes, int XB, int G, const uint32_t *alist) {
    const int lane = threadIdx.x & 31, A = W.arena, per_arena = A * (A - 1) / 2;
    const float reach = 2.f * W.rc, reach2 = reach * reach, kw2 = W.kw2, kc = W.kc;
    const float *X0 = reinterpret_cast<const float *>(xw);
    int start = 0;
    for (int pr = 0; pr < (G / A) * per_arena; ++pr) {
        const int end = __float_as_int(X0[XC_LH + 1 + pr]);
        if (end > start) {   // read from shared memory: the same on every lane
            int i = 0, t = pr % per_arena;
            while (t >= A - 1 - i) { t -= A - 1 - i; ++i; }
            const int gi = (pr / per_arena) * A + i, gj = gi + 1 + t;
            float *Xi = reinterpret_cast<float *>(xw + gi * XB);
            float *Xj = reinterpret_cast<float *>(xw + gj * XB);
            if (Xi[XC_ACTIVE] != 0.f && Xj[XC_ACTIVE] != 0.f) {
                float ci[3], Ri[9], vi[3], wi[3], cj[3], Rj[9], vj[3], wj[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    ci[k] = Xi[XC_C + k]; vi[k] = Xi[XC_V + k]; wi[k] = Xi[XC_W + k];
                    cj[k] = Xj[XC_C + k]; vj[k] = Xj[XC_V + k]; wj[k] = Xj[XC_W + k];
                }
#pragma unroll
                for (int k = 0; k < 9; ++k) { Ri[k] = Xi[XC_R + k]; Rj[k] = Xj[XC_R + k]; }
                const float4 *pti = reinterpret_cast<const float4 *>(pw + (ptrdiff_t)gi * sbytes);
                const float4 *ptj = reinterpret_cast<const float4 *>(pw + (ptrdiff_t)gj * sbytes);
                float fi[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, fj[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                for (int en = start + lane; en < end; en += 32) {
                    const uint32_t code = alist[en];
                    const float4 pa = pti[code & ((1u << AL_BITS) - 1u)], pb = ptj[code >> AL_BITS];
                    float ra[3], e[3];
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        ra[k] = Ri[3 * k] * pa.x + Ri[3 * k + 1] * pa.y + Ri[3 * k + 2] * pa.z;
                        e[k] = (ci[k] + ra[k]) - cj[k];
                    }
                    const float ah0 = Rj[0] * e[0] + Rj[3] * e[1] + Rj[6] * e[2];
                    const float ah1 = Rj[1] * e[0] + Rj[4] * e[1] + Rj[7] * e[2];
                    const float ah2 = Rj[2] * e[0] + Rj[5] * e[1] + Rj[8] * e[2];
                    const float d0 = ah0 - pb.x, d1 = ah1 - pb.y, d2 = ah2 - pb.z;
                    const float dd = d0 * d0 + d1 * d1 + d2 * d2;
                    if (dd < reach2 && dd > 0.f)
                        pair_force(pa, pb, ra, d0, d1, d2, dd, Rj, vi, wi, vj, wj, reach, kw2, kc, fi, fj);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
                    for (int k = 0; k < 6; ++k) {
                        fi[k] += __shfl_xor_sync(FULL_MASK, fi[k], o);
                        fj[k] += __shfl_xor_sync(FULL_MASK, fj[k], o);
                    }
                }
                if (lane == 0) {
#pragma unroll
                    for (int k = 0; k < 6; ++k) { Xi[XC_RF + k] += fi[k]; Xj[XC_RF + k] += fj[k]; }
                }
                __syncwarp();
            }
        }
        start = end;
    }
}

template <int LPS>
__device__ __forceinline__ void arena_wrench(const WorldDev &W, unsigned char *xch, int sbytes, const float4 *pts,
                                             int c0, int nc, int p0, int np, const float c[3], const float R[9],
                                             const float v[3], const float om[3], const float bbc[3],
                                             const float bbh[3], bool active, float rmax, bool fresh,
                                             uint32_t *alist, int gl, float (&rf)[6]) {
    constexpr int G = 32 / LPS;
    const int lane = threadIdx.x & 31, g = lane / LPS, A = W.arena, XB = xch_bytes(W.max_chunks);
    float *X = reinterpret_cast<float *>(xch);
    float4 *LW = reinterpret_cast<float4 *>(xch + 4 * XC_N);
    const float4 *LB = LW + 2 * W.max_chunks;
    // world boxes: all points (the body box turned by R) and each link
    float wc[3], wh[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        wc[i] = c[i] + (R[3 * i] * bbc[0] + R[3 * i + 1] * bbc[1] + R[3 * i + 2] * bbc[2]);
        wh[i] = fabsf(R[3 * i]) * bbh[0] + fabsf(R[3 * i + 1]) * bbh[1] + fabsf(R[3 * i + 2]) * bbh[2];
    }
    for (int l = gl; l < nc; l += LPS) {
        const float4 cb = LB[2 * l], hb = LB[2 * l + 1];
        LW[2 * l] = make_float4(c[0] + (R[0] * cb.x + R[1] * cb.y + R[2] * cb.z),
                                c[1] + (R[3] * cb.x + R[4] * cb.y + R[5] * cb.z),
                                c[2] + (R[6] * cb.x + R[7] * cb.y + R[8] * cb.z), 0.f);
        LW[2 * l + 1] = make_float4(fabsf(R[0]) * hb.x + fabsf(R[1]) * hb.y + fabsf(R[2]) * hb.z,
                                    fabsf(R[3]) * hb.x + fabsf(R[4]) * hb.y + fabsf(R[5]) * hb.z,
                                    fabsf(R[6]) * hb.x + fabsf(R[7]) * hb.y + fabsf(R[8]) * hb.z, 0.f);
    }
    if (gl == 0) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            X[XC_C + i] = c[i]; X[XC_V + i] = v[i]; X[XC_W + i] = om[i];
            X[XC_BC + i] = wc[i]; X[XC_BH + i] = wh[i];
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) X[XC_R + i] = R[i];
        X[XC_ACTIVE] = active ? 1.f : 0.f;
        X[XC_C0] = __int_as_float(c0);
        X[XC_NC] = __int_as_float(nc);
        X[XC_P0] = __int_as_float(p0);
        X[XC_NP] = __int_as_float(np);
    }
    if (gl < 6) X[XC_RF + gl] = 0.f;
    if (gl == 0) {   // how far the robot's points may have moved since the list was built
        float dc = 0.f, dr = 0.f;
#pragma unroll
        for (int i = 0; i < 3; ++i) dc += (c[i] - X[XC_CREF + i]) * (c[i] - X[XC_CREF + i]);
#pragma unroll
        for (int i = 0; i < 9; ++i) dr += (R[i] - X[XC_RREF + i]) * (R[i] - X[XC_RREF + i]);
        X[XC_D] = 1.0001f * (sqrtf(dc) + (0.70711f * sqrtf(dr) + 1e-5f) * rmax);
    }
    __syncwarp();
    const float reach = 2.f * W.rc, reach2 = reach * reach, cull = reach + ARENA_MARGIN;
    const float kw2 = W.kw2, kc = W.kc;
    unsigned char *xw = xch - g * XB;                                     // the warp's first area
    const unsigned char *pw = reinterpret_cast<const unsigned char *>(pts) - (ptrdiff_t)g * sbytes;  // first slot
    const int per_arena = A * (A - 1) / 2;
    if (alist) {
        // the pair list: rebuilt at a launch's first step, after joint updates and when two robots
        // of a pair may together have moved a skin (2 rc) since it was built
        float *X0 = reinterpret_cast<float *>(xw);
        const float skin = 2.f * W.rc;
        bool need = fresh || __float_as_int(X0[XC_LH]) == 0;
        for (int pr = 0; pr < (G / A) * per_arena; ++pr) {
            int i = 0, t = pr % per_arena;
            while (t >= A - 1 - i) { t -= A - 1 - i; ++i; }
            const int gi = (pr / per_arena) * A + i, gj = gi + 1 + t;
            const float *Xi = reinterpret_cast<const float *>(xw + gi * XB);
            const float *Xj = reinterpret_cast<const float *>(xw + gj * XB);
            need = need || Xi[XC_D] + Xj[XC_D] > skin;
        }
        if (need) {   // the same on every lane (fresh is; the rest is read from shared memory)
            if (gl == 0) {
#pragma unroll
                for (int i = 0; i < 3; ++i) X[XC_CREF + i] = c[i];
#pragma unroll
                for (int i = 0; i < 9; ++i) X[XC_RREF + i] = R[i];
            }
            __syncwarp();
            const int n = arena_build(W, xw, pw, sbytes, XB, G, reach + skin, alist);
            if (lane == 0) X0[XC_LH] = __int_as_float(n <= W.alist_cap ? 1 : 2);
            __syncwarp();
        }
        if (__float_as_int(X0[XC_LH]) == 1) {
            arena_list_forces(W, xw, pw, sbytes, XB, G, alist);
#pragma unroll
            for (int k = 0; k < 6; ++k) rf[k] = X[XC_RF + k];
            __syncwarp();   // the exchange area is written again next step
            return;
        }
    }
    for (int pr = 0; pr < (G / A) * per_arena; ++pr) {   // the same pairs, in the same order, on every lane
        int i = 0, t = pr % per_arena;
        while (t >= A - 1 - i) { t -= A - 1 - i; ++i; }
        const int gi = (pr / per_arena) * A + i, gj = gi + 1 + t;
        float *Xi = reinterpret_cast<float *>(xw + gi * XB);
        float *Xj = reinterpret_cast<float *>(xw + gj * XB);
        bool ov = Xi[XC_ACTIVE] != 0.f && Xj[XC_ACTIVE] != 0.f;
#pragma unroll
        for (int k = 0; k < 3; ++k) ov = ov && fabsf(Xi[XC_BC + k] - Xj[XC_BC + k]) <= Xi[XC_BH + k] + Xj[XC_BH + k] + cull;
        if (!ov) continue;   // read from shared memory: the same on every lane
        const float4 *LWi = reinterpret_cast<const float4 *>(xw + gi * XB + 4 * XC_N);
        const float4 *LWj = reinterpret_cast<const float4 *>(xw + gj * XB + 4 * XC_N);
        const float4 *LBj = LWj + 2 * W.max_chunks;
        uint64_t *NMi = reinterpret_cast<uint64_t *>(xw + gi * XB + 4 * XC_N + 64 * W.max_chunks);
        const int nli = __float_as_int(Xi[XC_NC]), nlj = __float_as_int(Xj[XC_NC]);
        const int p0i = __float_as_int(Xi[XC_P0]), npi = __float_as_int(Xi[XC_NP]);
        const int l0j = __float_as_int(Xj[XC_C0]);
        // chunks of j near each chunk of i (only chunks of i inside j's world box)
        const float4 bcj = make_float4(Xj[XC_BC], Xj[XC_BC + 1], Xj[XC_BC + 2], 0.f);
        const float4 bhj = make_float4(Xj[XC_BH], Xj[XC_BH + 1], Xj[XC_BH + 2], 0.f);
        for (int l = lane; l < nli; l += 32) {
            uint64_t nm = 0;
            const float4 ca = LWi[2 * l], ha = LWi[2 * l + 1];
            if (boxes_meet(ca, ha, bcj, bhj, cull))
                for (int lb = 0; lb < nlj; ++lb)
                    if (boxes_meet(ca, ha, LWj[2 * lb], LWj[2 * lb + 1], cull)) nm |= 1ull << lb;
            NMi[l] = nm;
        }
        __syncwarp();
        float ci[3], Ri[9], vi[3], wi[3], cj[3], Rj[9], vj[3], wj[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            ci[k] = Xi[XC_C + k]; vi[k] = Xi[XC_V + k]; wi[k] = Xi[XC_W + k];
            cj[k] = Xj[XC_C + k]; vj[k] = Xj[XC_V + k]; wj[k] = Xj[XC_W + k];
        }
#pragma unroll
        for (int k = 0; k < 9; ++k) { Ri[k] = Xi[XC_R + k]; Rj[k] = Xj[XC_R + k]; }
        const float4 *pti = reinterpret_cast<const float4 *>(pw + (ptrdiff_t)gi * sbytes);
        const float4 *ptj = reinterpret_cast<const float4 *>(pw + (ptrdiff_t)gj * sbytes);
        float fi[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, fj[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int ia = lane; ia < npi; ia += 32) {
            const uint64_t nm = NMi[W.pchunk[p0i + ia]];
            if (!nm) continue;
            const float4 pa = pti[ia];
            float ra[3], e[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                ra[k] = Ri[3 * k] * pa.x + Ri[3 * k + 1] * pa.y + Ri[3 * k + 2] * pa.z;
                e[k] = (ci[k] + ra[k]) - cj[k];
            }
            // the point in j's body frame, Rj^T (x_a - c_j): distances to j's points are then
            // differences of stored offsets
            const float ah0 = Rj[0] * e[0] + Rj[3] * e[1] + Rj[6] * e[2];
            const float ah1 = Rj[1] * e[0] + Rj[4] * e[1] + Rj[7] * e[2];
            const float ah2 = Rj[2] * e[0] + Rj[5] * e[1] + Rj[8] * e[2];
            for (uint64_t bm = nm; bm; bm &= bm - 1) {
                const int lb = __ffsll((long long)bm) - 1;
                // skip the chunk unless the point is within reach of its body-frame box
                const float4 cbh = LBj[2 * lb], hbh = LBj[2 * lb + 1];
                if (fabsf(ah0 - cbh.x) > hbh.x + cull || fabsf(ah1 - cbh.y) > hbh.y + cull ||
                    fabsf(ah2 - cbh.z) > hbh.z + cull)
                    continue;
                const int b1 = W.cpo[l0j + lb + 1];
#pragma unroll 4
                for (int ib = W.cpo[l0j + lb]; ib < b1; ++ib) {
                    const float4 pb = ptj[__ldg(W.lpt + ib)];
                    const float d0 = ah0 - pb.x, d1 = ah1 - pb.y, d2 = ah2 - pb.z;
                    const float dd = d0 * d0 + d1 * d1 + d2 * d2;
                    if (dd < reach2 && dd > 0.f)
                        pair_force(pa, pb, ra, d0, d1, d2, dd, Rj, vi, wi, vj, wj, reach, kw2, kc, fi, fj);
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                fi[k] += __shfl_xor_sync(FULL_MASK, fi[k], o);
                fj[k] += __shfl_xor_sync(FULL_MASK, fj[k], o);
            }
        }
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < 6; ++k) { Xi[XC_RF + k] += fi[k]; Xj[XC_RF + k] += fj[k]; }
        }
        __syncwarp();
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) rf[k] = X[XC_RF + k];
    __syncwarp();   // the exchange area is written again next step
}

// ------------------------------------------------------------------------ one scene, n steps

// OPT: the friction-model options (W.fric_mode) are compiled in; without them the step is the
// least squares of Eqs. 1-6 as written, with no test of the options in the step loop; ARENA:
// robot-robot contact within arenas (below)
template <int LPS, bool FLAT, bool OPT, bool ARENA>
__device__ void run_scene(const WorldDev &W, int s, int gl, float4 *pts, float *fr, float *th,
                          float *th_old, float4 *tb, int n_steps, long long step0, unsigned char *xch,
                          int sbytes, const CUtensorMap *tmap, int item) {
    const bool valid = s >= 0;
    int p0 = 0, np = 0, l0 = 0, nl = 1;
    if (valid) {
        p0 = W.point_off[s]; np = W.point_off[s + 1] - p0;
        l0 = W.link_off[s]; nl = W.link_off[s + 1] - l0;
    }
    const int j0 = l0 - (valid ? s : 0), nj = nl - 1;
    // ---- load
    float c[3], q[4], v[3], L[3];
    uint32_t status = 1u;
    float mu = 0.f;
    int hm = -1;
    if (valid) {
        const int S = W.S;
        c[0] = W.st[ST_CX * S + s]; c[1] = W.st[ST_CY * S + s]; c[2] = W.st[ST_CZ * S + s];
        q[0] = W.st[ST_QW * S + s]; q[1] = W.st[ST_QX * S + s]; q[2] = W.st[ST_QY * S + s];
        q[3] = W.st[ST_QZ * S + s];
        v[0] = W.st[ST_VX * S + s]; v[1] = W.st[ST_VY * S + s]; v[2] = W.st[ST_VZ * S + s];
        L[0] = W.st[ST_LX * S + s]; L[1] = W.st[ST_LY * S + s]; L[2] = W.st[ST_LZ * S + s];
        status = W.status[s];
        mu = W.mu[s];
        hm = FLAT ? -1 : W.hmap[s];
    } else {
        c[0] = c[1] = c[2] = 0.f; q[0] = 1.f; q[1] = q[2] = q[3] = 0.f;
        v[0] = v[1] = v[2] = 0.f; L[0] = L[1] = L[2] = 0.f;
    }
    for (int j = gl; j < nj; j += LPS) th[j] = W.theta[j0 + j];
    uint64_t kprev = 0;
    if (!W.reseed) {
#pragma unroll 8
        for (int k = 0, i = gl; i < np; ++k, i += LPS)
            if (W.kappa[p0 + i]) kprev |= 1ull << k;
    }
    __syncwarp();
    Shape sh;
    float rmax;
    // the posed shape of the current joint angles: read from the posed-shape cache when the
    // launch says every entry is current, else rebuilt (and written to the cache when there is one)
    if (!ARENA && W.scache_mode == 2) {
        rmax = scache_load<LPS>(W, valid ? s : -1, np, pts, tb, sh, gl);
    } else {
        shape_update<LPS>(W, valid ? s : 0, p0, np, l0, nl, th, fr, pts, gl, sh);
        rmax = tile_bounds<LPS>(pts, np, tb, gl);
        if (!ARENA && W.scache_mode != 0 && valid) scache_store<LPS>(W, s, np, pts, tb, sh, rmax, fr, l0, nl, gl);
    }
    // (arenas) body-frame box of the posed points
    float bbc[3] = {0.f, 0.f, 0.f}, bbh[3] = {0.f, 0.f, 0.f};
    float4 *lbb = reinterpret_cast<float4 *>(xch + 4 * XC_N) + 2 * W.max_chunks;   // body chunk boxes
    int c0 = 0, nc = 0;   // (arenas) the scene's broad-phase chunks
    if (ARENA) {
        if (valid) { c0 = W.coff[s]; nc = W.coff[s + 1] - c0; }
        robot_box<LPS>(tb, (np + LPS - 1) / LPS, gl, bbc, bbh);
        chunk_boxes_body<LPS>(W, c0, nc, fr, sh.g, lbb, gl);
    }
    if (W.reseed) {
        // the previous-step contacts from a detection at the current state (same test as the
        // step's own: z below the ground at the point's cell)
        float R0[9];
        quat_mat(q, R0);
        for (int k = 0, i = gl; i < np; ++k, i += LPS) {
            const float4 r = pts[i];
            const float x = c[0] + (R0[0] * r.x + R0[1] * r.y + R0[2] * r.z);
            const float y = c[1] + (R0[3] * r.x + R0[4] * r.y + R0[5] * r.z);
            const float z = c[2] + (R0[6] * r.x + R0[7] * r.y + R0[8] * r.z);
            if (z < ground<FLAT>(W, hm, x, y)) kprev |= 1ull << k;
        }
    }
    // sh is written by the (out-of-line) shape update through a reference, so it lives in local
    // memory; the step loop reads this register copy
    Shape shr = sh;
    // highest ground a point can meet (plus a margin for the rounding of the bound)
    const float hmax = (FLAT || hm < 0 ? 0.f : W.hm_max[hm]) + 1e-5f;
    // (height maps) the ground bound of the cull: the map's highest cell, or, while the scene's
    // points all lie within hm_dr cells of its CoG's cell at the last cull, the dilated map's
    // entry there (local: in use; dm_lim: the largest posed radius plus drift that keeps it valid)
    const bool dm = !FLAT && hm >= 0 && W.hm_dmax != nullptr;
    const float dm_lim = dm ? ((float)W.hm_dr - 1.5f) / W.hm_scale : 0.f;
    float hcull = hmax, cull_x = 0.f, cull_y = 0.f;
    bool local = false;
    // height-map window (after the slot); its origin is negative until the first refresh.  With
    // TMA the window's first cell sits wsh cells into each stored row; its mbarrier follows it.
    float *win = reinterpret_cast<float *>(reinterpret_cast<unsigned char *>(pts) +
                                           hm_win_offset(W.max_points, W.max_links, LPS));
    uint64_t *wbar = reinterpret_cast<uint64_t *>(win + HM_BOX * HM_WIN);
    int wx0 = -(1 << 24), wy0 = -(1 << 24), wsh = 0;
    uint32_t wphase = 0;
    bool wfail = false;
    const bool win_tma = !FLAT && W.hm_tma != 0;
    if (win_tma) {
        if (gl == 0) win_bar_init(wbar);
        __syncwarp();
    }
    const int ntiles = (np + LPS - 1) / LPS;

    const float dt = W.dt, idt = 1.0f / W.dt, kw2 = W.kw2, kc = W.kc;
    // friction-model options (Sec. III-C, the refinements named after Eq. 6): rows weighted by
    // the normal forces; the friction impulse's torque about the horizontal axes
    const bool weighted = OPT && (W.fric_mode & 1) != 0, tilt = OPT && (W.fric_mode & 2) != 0;
    float iM = 1.0f / shr.M;
    const bool actuated = W.act_mode != 0;
    // Candidate tiles: those whose box came within CULL_MARGIN of the highest ground at the last
    // cull.  slack is the height above the highest ground of the lowest box left out then, minus
    // a bound on how far any point has moved down since
    // (integration only: the friction corrections move the robot horizontally and rotate it about
    // the vertical); while it is >= 0 no other tile can have reached the ground, so the set stays
    // exact and the boxes are tested again only when it runs out or the shape changes.
    float slack = -1.f;
    uint64_t cand = 0;
    int ph = (int)(step0 % (long long)W.K);
    for (int t = 0; t < n_steps; ++t) {
        const long long n = step0 + t;
        const bool tick = actuated && ph == 0;
        ph = (ph + 1 == W.K) ? 0 : ph + 1;
        float R[9];
        quat_mat(q, R);

        // -- joint-angle determination: new angles, frames, mass properties and offsets; the
        //    old angles and CoG are kept for the kinematic slip of the contact points
        float gold[3] = {0.f, 0.f, 0.f};
        if (tick) {
            gold[0] = shr.g[0]; gold[1] = shr.g[1]; gold[2] = shr.g[2];
            const bool gp = W.act_mode == 2;
            if (gp) {
                // the controller reads the foot contacts of the last step and sets the targets
                uint32_t sens = 0;
                for (int k = 0, i = gl; i < np; ++k, i += LPS)
                    if ((kprev >> k) & 1ull) {
                        const int sid = W.links[l0 + W.plink[p0 + i]].sensor;
                        if (sid >= 0 && sid < 32) sens |= 1u << sid;
                    }
                sens = gor<LPS>(sens);
                if (gl == 0 && valid && status == 0u) gp_run(W, s, j0, nj, sens);
                __syncwarp();
            }
            for (int j = gl; j < nj; j += LPS) {
                th_old[j] = th[j];
                if (status == 0u) {   // a frozen scene keeps its angles
                    const LinkDev lk = W.links[l0 + j + 1];
                    const float tgt = gp ? (float)W.gp_k[j0 + j] * GP_STEP : joint_target(W, j0 + j, n);
                    th[j] = fminf(fmaxf(tgt, lk.lo), lk.hi);
                }
            }
            __syncwarp();
            shape_update<LPS>(W, valid ? s : 0, p0, np, l0, nl, th, fr, pts, gl, sh);
            rmax = tile_bounds<LPS>(pts, np, tb, gl);
            if (!ARENA && W.scache_mode != 0 && valid) scache_store<LPS>(W, s, np, pts, tb, sh, rmax, fr, l0, nl, gl);
            shr = sh;
            if (ARENA) {
                robot_box<LPS>(tb, ntiles, gl, bbc, bbh);
                chunk_boxes_body<LPS>(W, c0, nc, fr, shr.g, lbb, gl);
            }
            iM = 1.0f / shr.M;
            slack = -1.f;   // the tiles moved: cull again
        }

        float om[3];
        world_sym(R, shr.Ii, L, om);

        // -- (arenas) contact forces and their torques about the CoG from the other robots
        float rf[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (ARENA)
            arena_wrench<LPS>(W, xch, sbytes, pts, c0, nc, p0, np, c, R, v, om, bbc, bbh, valid && status == 0u,
                              rmax, t == 0 || tick, W.alist ? W.alist + (size_t)item * W.alist_cap : nullptr, gl, rf);

        // -- pass 1: collision against the ground and penalty normal forces over the candidate
        //    tiles.  For the points in contact in both steps (the friction set C, Sec. III-C) it
        //    also sums the count, the first and the second moments of d = rho - o, rho = R r,
        //    about a reference point o near them: every term of the dynamic least squares is a
        //    function of these (see below).  All sums are independent, so the group reduction is
        //    one butterfly and every lane ends with bit-identical values.
        if (!FLAT) {
            // move the height-map window when the origin that would centre it on the CoG's cell
            // (clamped to the map) has drifted from the current one by more than HM_DRIFT cells;
            // a window held at the map's edge stays put (the groups of the warp refresh together;
            // each loads only its own window)
            const int cx = __float2int_rd(__fmul_rn(__fsub_rn(c[0], W.hm_ox), W.hm_scale));
            const int cy = __float2int_rd(__fmul_rn(__fsub_rn(c[1], W.hm_oy), W.hm_scale));
            const int tx = min(max(cx - HM_WIN / 2, 0), max(W.hm_nx - HM_WIN, 0));
            const int ty = min(max(cy - HM_WIN / 2, 0), max(W.hm_ny - HM_WIN, 0));
            const bool need = hm >= 0 && (wx0 < 0 || abs(tx - wx0) > HM_DRIFT || abs(ty - wy0) > HM_DRIFT);
            if (__any_sync(FULL_MASK, need)) {
                // with TMA: one lane of each group that moves its window issues one box of the
                // map (16 x 16 cells here: maps with TMA are at least that large, so the window
                // lies inside the map), x rounded down to a multiple of 4 cells; columns past the
                // map's edge, outside the window, read as zero and are never looked up.  The
                // warp meets after the copies are issued and waits for them as one.
                const bool tma = need && win_tma && !wfail;
                if (need) {
                    wx0 = tx;
                    wy0 = ty;
                    wsh = tma ? wx0 - (wx0 & ~3) : 0;
                    if (tma && gl == 0) win_load(win, tmap, wx0 & ~3, wy0, hm, wbar);
                }
                __syncwarp();
                const bool landed = win_wait_warp(wbar, wphase, tma);
                if (tma) {
                    wphase ^= 1u;
                    if (!landed) {   // the load gave up its bounded wait: freeze the scene
                        wfail = true;
                        status |= 4u;
                    }
                } else if (need && !wfail) {
                    const float *map = W.hm + (size_t)hm * W.hm_ny * W.hm_nx;
                    for (int e = gl; e < HM_WIN * HM_WIN; e += LPS) {
                        const int iy = wy0 + e / HM_WIN, ix = wx0 + e % HM_WIN;
                        win[(e / HM_WIN) * HM_BOX + e % HM_WIN] =
                            __ldg(map + (size_t)min(iy, W.hm_ny - 1) * W.hm_nx + min(ix, W.hm_nx - 1));
                    }
                }
                __syncwarp();
            }
        }
        // a local ground bound holds while every point is within hm_dr cells of the cull's cell:
        // |x - c_cull| <= rmax + |c - c_cull| (max norm; the rotation keeps |R p| <= rmax), and
        // clamping a cell index to the map moves it no further from the clamped centre
        if (!FLAT && local && rmax + fmaxf(fabsf(c[0] - cull_x), fabsf(c[1] - cull_y)) > dm_lim) slack = -1.f;
        // the cull's ballots involve the whole warp: every group culls when any one needs to
        if (__any_sync(FULL_MASK, slack < 0.f)) {
            if (!FLAT) {
                local = dm && rmax <= dm_lim;
                hcull = hmax;
                if (local) {
                    cull_x = c[0];
                    cull_y = c[1];
                    const int ix = min(max(__float2int_rd(__fmul_rn(__fsub_rn(c[0], W.hm_ox), W.hm_scale)), 0), W.hm_nx - 1);
                    const int iy = min(max(__float2int_rd(__fmul_rn(__fsub_rn(c[1], W.hm_oy), W.hm_scale)), 0), W.hm_ny - 1);
                    hcull = fminf(hmax, __ldg(W.hm_dmax + ((size_t)hm * W.hm_ny + iy) * W.hm_nx + ix) + 1e-5f);
                }
            }
            // the slack is the height of the lowest tile left out above the ground bound (at
            // least CULL_MARGIN; unbounded when no tile is left out)
            float zfar;
            cand = tiles_near_ground<LPS>(tb, ntiles, R, c[2], hcull + CULL_MARGIN, gl, zfar);
            slack = fminf(zfar - hcull, 1e30f);
        }
        // reference o of the friction-set moments: the rotated centre of the first tile holding a
        // point that was in contact last step (C is a subset of those; o depends on the state alone)
        int kf = kprev ? __ffsll((long long)kprev) - 1 : 64;
#pragma unroll
        for (int ofs = LPS / 2; ofs > 0; ofs >>= 1) kf = min(kf, __shfl_xor_sync(FULL_MASK, kf, ofs));
        float o[3] = {0.f, 0.f, 0.f};
        if (kf < 64) {
            const float4 lo = tb[2 * kf], hi = tb[2 * kf + 1];
            const float mid[3] = {0.5f * (lo.x + hi.x), 0.5f * (lo.y + hi.y), 0.5f * (lo.z + hi.z)};
            mat_vec(R, mid, o);
        }
        // FN, tau_x, tau_y | n | sum d (3) | sum d d^T (xx yy zz xy xz yz)
        float acc[13] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        // The 64-bit tile masks are walked as two 32-bit words (hexapod candidates sit in the low
        // word: points are stored by construction height).  Two tiles per iteration: two
        // independent chains; a point that is absent, not in contact or not in C adds an exact
        // zero, so the sums see the same terms in the same order.
        uint32_t knw[2] = {0u, 0u};
#pragma unroll
        for (int hw = 0; hw < 2; ++hw) {
            const uint32_t kp = (uint32_t)(kprev >> (32 * hw));
            for (uint32_t tm = (uint32_t)(cand >> (32 * hw)); tm;) {
                const int ja = __ffs(tm) - 1;
                tm &= tm - 1;
                const bool two = tm != 0;
                const int jb = two ? __ffs(tm) - 1 : ja;
                if (two) tm &= tm - 1;
                const int ia = gl + (ja + 32 * hw) * LPS, ib = gl + (jb + 32 * hw) * LPS;
                const bool oka = ia < np, okb = two && ib < np;
                const float4 pa = pts[oka ? ia : 0], pb = pts[okb ? ib : 0];
                const float rxa = R[0] * pa.x + R[1] * pa.y + R[2] * pa.z, rxb = R[0] * pb.x + R[1] * pb.y + R[2] * pb.z;
                const float rya = R[3] * pa.x + R[4] * pa.y + R[5] * pa.z, ryb = R[3] * pb.x + R[4] * pb.y + R[5] * pb.z;
                const float rza = R[6] * pa.x + R[7] * pa.y + R[8] * pa.z, rzb = R[6] * pb.x + R[7] * pb.y + R[8] * pb.z;
                const float za = c[2] + rza, zb = c[2] + rzb;
                const float ha = ground_win<FLAT>(W, hm, win + wsh, wx0, wy0, c[0] + rxa, c[1] + rya);
                const float hb = ground_win<FLAT>(W, hm, win + wsh, wx0, wy0, c[0] + rxb, c[1] + ryb);
                const bool ca = oka && za < ha, cb = okb && zb < hb;
                const float vza = v[2] + (om[0] * rya - om[1] * rxa), vzb = v[2] + (om[0] * ryb - om[1] * rxb);
                const float Fa = ca ? fmaxf(0.f, pa.w * (kw2 * (ha - za) - kc * vza)) : 0.f;
                const float Fb = cb ? fmaxf(0.f, pb.w * (kw2 * (hb - zb) - kc * vzb)) : 0.f;
                knw[hw] |= (ca ? 1u << ja : 0u) | (cb ? 1u << jb : 0u);
                acc[0] += Fa; acc[1] += rya * Fa; acc[2] -= rxa * Fa;
                acc[0] += Fb; acc[1] += ryb * Fb; acc[2] -= rxb * Fb;
                // friction set C: in contact now and last step; a row's weight is 1, or its normal
                // force with force-weighted friction.  Sums: weight, weight x d, weight x d d^T
                const float wa = (ca && ((kp >> ja) & 1u)) ? (weighted ? Fa : 1.f) : 0.f;
                const float wb = (cb && ((kp >> jb) & 1u)) ? (weighted ? Fb : 1.f) : 0.f;
                const float da0 = rxa - o[0], da1 = rya - o[1], da2 = rza - o[2];
                const float db0 = rxb - o[0], db1 = ryb - o[1], db2 = rzb - o[2];
                const float a0 = wa * da0, a1 = wa * da1, a2 = wa * da2;
                const float b0 = wb * db0, b1 = wb * db1, b2 = wb * db2;
                acc[3] += wa; acc[3] += wb;
                acc[4] += a0; acc[5] += a1; acc[6] += a2;
                acc[4] += b0; acc[5] += b1; acc[6] += b2;
                acc[7] += a0 * da0; acc[8] += a1 * da1; acc[9] += a2 * da2;
                acc[10] += a0 * da1; acc[11] += a0 * da2; acc[12] += a1 * da2;
                acc[7] += b0 * db0; acc[8] += b1 * db1; acc[9] += b2 * db2;
                acc[10] += b0 * db1; acc[11] += b0 * db2; acc[12] += b1 * db2;
            }
        }
        const uint64_t know = (uint64_t)knw[0] | ((uint64_t)knw[1] << 32);
        gsum<LPS, 13>(acc);
        const float FN = acc[0];
        // friction set: count, centroid of rho and second central moments sum (rho - gb)(rho - gb)^T
        const float nC = acc[3];
        const float in = nC > 0.f ? __fdividef(1.f, nC) : 0.f;
        const float e0 = acc[4] * in, e1 = acc[5] * in, e2 = acc[6] * in;   // centroid - o
        const float gb[3] = {o[0] + e0, o[1] + e1, o[2] + e2};
        const Sym M2 = {acc[7] - nC * (e0 * e0), acc[8] - nC * (e1 * e1), acc[9] - nC * (e2 * e2),
                        acc[10] - nC * (e0 * e1), acc[11] - nC * (e0 * e2), acc[12] - nC * (e1 * e2)};

        // -- semi-implicit Euler
        float vs[3], Ls[3], cs[3], qs[4], oms[3];
        vs[0] = v[0] + dt * W.gx;
        vs[1] = v[1] + dt * W.gy;
        vs[2] = v[2] + dt * (W.gz + FN * iM);
        Ls[0] = L[0] + dt * acc[1];
        Ls[1] = L[1] + dt * acc[2];
        Ls[2] = L[2];
        if (ARENA) {
            vs[0] += dt * (rf[0] * iM); vs[1] += dt * (rf[1] * iM); vs[2] += dt * (rf[2] * iM);
            Ls[0] += dt * rf[3]; Ls[1] += dt * rf[4]; Ls[2] += dt * rf[5];
        }
        world_sym(R, shr.Ii, Ls, oms);
        cs[0] = c[0] + dt * vs[0]; cs[1] = c[1] + dt * vs[1]; cs[2] = c[2] + dt * vs[2];
        // rotation increment dR = exp([u]x), u = dt w*: q* = dq (x) q and R* = dR R, so a point's
        // offset moves from rho to (1 + D) rho with D = dR - 1 = a [u]x + b [u]x^2
        // (a = sin|u| / |u|, b = (1 - cos|u|) / |u|^2), free of the cancellation in R* r - R r
        float Dm[6];   // rows 0 and 1 of D (only horizontal displacements are needed)
        float rzc = 0.f;   // (with the horizontal-axis friction torque) height of the integrated
                           // friction-set centroid above the integrated CoG: [(1 + D) gb]_z
        {
            const float px = dt * oms[0], py = dt * oms[1], pz = dt * oms[2];
            const float a2 = px * px + py * py + pz * pz;
            const float ra = a2 > 0.f ? rsqrtf(a2) : 0.f;   // 1 / |u|
            const float a = a2 * ra;
            float dq[4] = {1.f, 0.f, 0.f, 0.f};
            float fa = 1.f, fb = 0.5f;
            if (a > 0.f) {
                float sn, cn;
                sincos_small(0.5f * a, &sn, &cn);
                const float f = sn * ra;
                dq[0] = cn; dq[1] = f * px; dq[2] = f * py; dq[3] = f * pz;
                fa = 2.f * f * cn;
                fb = 2.f * f * f;
            }
            if (tilt)
                rzc = gb[2] + (-fa * py + fb * pz * px) * gb[0] + (fa * px + fb * pz * py) * gb[1] +
                      fb * (pz * pz - a2) * gb[2];
            // [u]x^2 = u u^T - |u|^2 1
            Dm[0] = fb * (px * px - a2); Dm[1] = -fa * pz + fb * px * py; Dm[2] = fa * py + fb * px * pz;
            Dm[3] = fa * pz + fb * py * px; Dm[4] = fb * (py * py - a2); Dm[5] = -fa * px + fb * py * pz;
            quat_mul(dq, q, qs);
            const float inv = rsqrtf(qs[0] * qs[0] + qs[1] * qs[1] + qs[2] * qs[2] + qs[3] * qs[3]);
            qs[0] *= inv; qs[1] *= inv; qs[2] *= inv; qs[3] *= inv;
            // largest downward move of any point this step: dt max(0, -v*_z) from the CoG plus the
            // rotation's: for x = R r, ((dR - 1) x)_z = sin|u| (n x x)_z + (1 - cos|u|) (n (n.x) - x)_z
            // with n = u / |u|, so |dz| <= (|u_xy| + |u|^2 / 2) |x| (yaw moves no point up or
            // down; |u_xy| <= |u_x| + |u_y|); a small factor covers rounding
            slack -= fmaxf(0.f, -dt * vs[2]) + 1.0001f * (fabsf(px) + fabsf(py) + 0.5f * a2) * rmax;
        }

        // -- friction (Sec. III-C, Eqs. 1-6) over C.  With d_i = rho_i - centroid and
        //    M2 = sum d d^T, the integrated sources are s_i = [(1 + D) rho_i]_xy and the slips
        //    e_i = -dt v*_xy - [D rho_i]_xy, so about the source centroid
        //      S2 = a_x^T M2 a_x + a_y^T M2 a_y,  sum s~ x e = -(a_x^T M2 b_y - a_y^T M2 b_x),
        //      mean e = -dt v*_xy - [D centroid]_xy
        //    with a_x, a_y the x, y rows of (1 + D) and b_x, b_y those of D.
        float cn[3] = {cs[0], cs[1], cs[2]}, vn[3] = {vs[0], vs[1], vs[2]};
        float Ln[3] = {Ls[0], Ls[1], Ls[2]}, qn[4] = {qs[0], qs[1], qs[2], qs[3]};
        // kinematic least squares (joint-update steps): a second pass over C about the exact
        // centroid of the moved points, slip R (r_old - r_new) back to the step start
        float f6[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (tick) {
            // old frames again (the new ones are no longer needed this step)
            link_frames<LPS>(W, l0, nl, th_old, fr, gl);
            for (uint64_t cm = kprev & know; cm; cm &= cm - 1) {
                const int k = __ffsll((long long)cm) - 1;
                const int i = gl + k * LPS;
                const float4 r = pts[i];
                const float4 a0 = W.p0m[p0 + i];
                float po[3];
                fk_point(fr, a0, W.plink[p0 + i], po);
                const float4 ro = make_float4(po[0] - gold[0], po[1] - gold[1], po[2] - gold[2], 0.f);
                const float rx = R[0] * r.x + R[1] * r.y + R[2] * r.z;
                const float ry = R[3] * r.x + R[4] * r.y + R[5] * r.z;
                const float ux = rx - gb[0];
                const float uy = ry - gb[1];
                const float d[3] = {ro.x - r.x, ro.y - r.y, ro.z - r.z};
                const float kx = R[0] * d[0] + R[1] * d[1] + R[2] * d[2];
                const float ky = R[3] * d[0] + R[4] * d[1] + R[5] * d[2];
                float wk = 1.f;   // the row's weight: its normal force this step (as in pass 1)
                if (weighted) {
                    const float rz = R[6] * r.x + R[7] * r.y + R[8] * r.z;
                    const float z = c[2] + rz;
                    const float h = ground_win<FLAT>(W, hm, win + wsh, wx0, wy0, c[0] + rx, c[1] + ry);
                    const float vz = v[2] + (om[0] * ry - om[1] * rx);
                    wk = fmaxf(0.f, r.w * (kw2 * (h - z) - kc * vz));
                }
                const float wux = wk * ux, wuy = wk * uy;
                f6[0] += wux; f6[1] += wuy; f6[2] += wux * ux + wuy * uy;
                f6[3] += wk * kx; f6[4] += wk * ky; f6[5] += wux * ky - wuy * kx;
            }
            gsum<LPS, 6>(f6);
        }
        if (nC > 0.f) {
            const float ax[3] = {1.f + Dm[0], Dm[1], Dm[2]}, ay[3] = {Dm[3], 1.f + Dm[4], Dm[5]};
            const float bx[3] = {Dm[0], Dm[1], Dm[2]}, by[3] = {Dm[3], Dm[4], Dm[5]};
            float Max[3], May[3];
            sym_mul(M2, ax, Max);
            sym_mul(M2, ay, May);
            const float S2 = ax[0] * Max[0] + ax[1] * Max[1] + ax[2] * Max[2] +
                             ay[0] * May[0] + ay[1] * May[1] + ay[2] * May[2];
            const float X = -((Max[0] * by[0] + Max[1] * by[1] + Max[2] * by[2]) -
                              (May[0] * bx[0] + May[1] * bx[1] + May[2] * bx[2]));
            const float sbx = ax[0] * gb[0] + ax[1] * gb[1] + ax[2] * gb[2];  // source centroid - c*
            const float sby = ay[0] * gb[0] + ay[1] * gb[1] + ay[2] * gb[2];
            const float tDx = -dt * vs[0] - (bx[0] * gb[0] + bx[1] * gb[1] + bx[2] * gb[2]);
            const float tDy = -dt * vs[1] - (by[0] * gb[0] + by[1] * gb[1] + by[2] * gb[2]);
            // a rotation needs two distinct points (force-weighted: a weighted mean spread about
            // the centre of pressure above 1e-6 m^2, far above the rounding left by the moments'
            // cancellation when the weight sits on one point)
            float a3 = (weighted ? S2 > 1e-6f * nC : (nC >= 2.f && S2 > 1e-12f)) ? __fdividef(X, S2) : 0.f;
            a3 = fminf(fmaxf(a3, -1.f), 1.f);
            const float t1 = fmaxf(0.f, 1.f - a3 * a3);
            const float cD = t1 > 0.f ? t1 * rsqrtf(t1) : 0.f;       // cos(alpha_D)
            const float r1 = __fdividef(1.f, 1.f + cD);
            const float cm1 = -a3 * a3 * r1;                          // cos(alpha_D) - 1
            const float dDx = -sbx, dDy = -sby;                       // CoG minus centroid
            const float DDx = tDx + cm1 * dDx - a3 * dDy;             // uncapped CoG shift
            const float DDy = tDy + a3 * dDx + cm1 * dDy;
            // maximum static friction (Coulomb cap on the impulse that undoes the slip)
            const float sh2 = 0.5f * a3 * a3 * r1;                    // sin^2(alpha_D / 2)
            const float u2 = tDx * tDx + tDy * tDy + 4.f * sh2 * S2 * in;
            const float Jreq = shr.M * (u2 > 0.f ? u2 * rsqrtf(u2) : 0.f) * idt;
            const float Jmax = mu * dt * FN;
            const float sc = (Jreq <= Jmax) ? 1.f : __fdividef(Jmax, Jreq);
            const float aD = asin_small(a3);
            float s1, c1;
            sincos_small(0.5f * sc * aD, &s1, &c1);
            const float sin1 = 2.f * s1 * c1, cm1s = -2.f * s1 * s1;
            float dx1 = sc * tDx + cm1s * dDx - sin1 * dDy;
            float dy1 = sc * tDy + sin1 * dDx + cm1s * dDy;
            float A = sc * aD;
            if (tick) {
                const float kbx = f6[0] * in, kby = f6[1] * in;
                const float S2K = f6[2] - nC * (kbx * kbx + kby * kby);
                const float tKx = f6[3] * in, tKy = f6[4] * in;
                const float XK = f6[5] - (kbx * f6[4] - kby * f6[3]);
                float a3K = (weighted ? S2K > 1e-6f * nC : (nC >= 2.f && S2K > 1e-12f)) ? __fdividef(XK, S2K) : 0.f;
                a3K = fminf(fmaxf(a3K, -1.f), 1.f);
                const float aK = asin_small(a3K);
                float s2, c2;
                sincos_small(0.5f * aK, &s2, &c2);
                const float sin2 = 2.f * s2 * c2, cm2 = -2.f * s2 * s2;
                // moved-point centroid is c + gb + kb; CoG after the dynamic map is cs + d1
                const float dKx = (cs[0] - c[0]) + dx1 - (gb[0] + kbx);
                const float dKy = (cs[1] - c[1]) + dy1 - (gb[1] + kby);
                dx1 += tKx + cm2 * dKx - sin2 * dKy;
                dy1 += tKy + sin2 * dKx + cm2 * dKy;
                A += aK;
            }
            cn[0] = cs[0] + dx1;
            cn[1] = cs[1] + dy1;
            vn[0] = vs[0] + sc * DDx * idt;
            vn[1] = vs[1] + sc * DDy * idt;
            // angular momentum of the yaw correction: (sc alpha_D / dt) R* Ib R*^T z
            float Rs[9];
            quat_mat(qs, Rs);
            const float ez[3] = {0.f, 0.f, 1.f};
            float Iz[3];
            world_sym(Rs, shr.Ib, ez, Iz);
            const float w = sc * aD * idt;
            Ln[0] = Ls[0] + w * Iz[0]; Ln[1] = Ls[1] + w * Iz[1]; Ln[2] = Ls[2] + w * Iz[2];
            if (tilt) {
                // the friction impulse J = M (v_new - v*) acts at the friction-set centroid,
                // rzc below the CoG: the x and y components of its moment r x J
                const float Jx = shr.M * (vn[0] - vs[0]), Jy = shr.M * (vn[1] - vs[1]);
                Ln[0] -= rzc * Jy;
                Ln[1] += rzc * Jx;
            }
            float sa, ca;
            sincos_small(0.5f * A, &sa, &ca);
            const float qz[4] = {ca, 0.f, 0.f, sa};
            quat_mul(qz, qs, qn);
        }

        // -- freeze a scene whose state is no longer finite or has left any sane range
        if (status == 0u) {
            // any NaN or infinity makes the sum non-finite (all terms are bounded below 1e6
            // in magnitude when finite, so the sum itself cannot overflow)
            const float chk = cn[0] + cn[1] + cn[2] + vn[0] + vn[1] + vn[2] + Ln[0] + Ln[1] +
                              Ln[2] + qn[0] + qn[1] + qn[2] + qn[3];
            const bool fin = isfinite(chk);
            if (!fin) {
                status |= 1u;
            } else if (fabsf(vn[0]) > 1e3f || fabsf(vn[1]) > 1e3f || fabsf(vn[2]) > 1e3f ||
                       fabsf(cn[0]) > 1e6f || fabsf(cn[1]) > 1e6f || fabsf(cn[2]) > 1e6f) {
                status |= 2u;
            } else {
#pragma unroll
                for (int i = 0; i < 3; ++i) { c[i] = cn[i]; v[i] = vn[i]; L[i] = Ln[i]; }
#pragma unroll
                for (int i = 0; i < 4; ++i) q[i] = qn[i];
                kprev = know;
            }
        }
    }

    if (win_tma) {
        win_wait_warp(wbar, wphase ^ 1u, wfail);   // a load that outlived its wait lands first
        __syncwarp();
        if (gl == 0) win_bar_inval(wbar);
        __syncwarp();
    }

    // ---- write back (contact sensors from the last step's contacts)
    uint32_t sens = 0;
    for (int k = 0, i = gl; i < np; ++k, i += LPS) {
        const uint8_t kb = (uint8_t)((kprev >> k) & 1ull);
        W.kappa[p0 + i] = kb;
        if (kb) {
            const int sid = W.links[l0 + W.plink[p0 + i]].sensor;
            if (sid >= 0 && sid < 32) sens |= 1u << sid;
        }
    }
    sens = gor<LPS>(sens);
    for (int j = gl; j < nj; j += LPS) W.theta[j0 + j] = th[j];
    if (valid && gl == 0) {
        const int S = W.S;
        W.st[ST_CX * S + s] = c[0]; W.st[ST_CY * S + s] = c[1]; W.st[ST_CZ * S + s] = c[2];
        W.st[ST_QW * S + s] = q[0]; W.st[ST_QX * S + s] = q[1]; W.st[ST_QY * S + s] = q[2];
        W.st[ST_QZ * S + s] = q[3];
        W.st[ST_VX * S + s] = v[0]; W.st[ST_VY * S + s] = v[1]; W.st[ST_VZ * S + s] = v[2];
        W.st[ST_LX * S + s] = L[0]; W.st[ST_LY * S + s] = L[1]; W.st[ST_LZ * S + s] = L[2];
        float R[9], om[3];
        quat_mat(q, R);
        world_sym(R, shr.Ii, L, om);
        W.omega[s] = om[0]; W.omega[S + s] = om[1]; W.omega[2 * S + s] = om[2];
        W.sensors[s] = sens;
        W.status[s] = status;
    }
    __syncwarp();
}

template <int LPS, bool FLAT, bool OPT, bool ARENA>
__device__ __forceinline__ void step_body(const WorldDev &W, int n_steps, int sbytes, const CUtensorMap *tmap) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // (height maps) a 128-byte aligned base, so that every window is aligned for its TMA box
    // (an integer offset from the shared array, so the pointer stays a shared-memory one)
    unsigned char *smem = smem_raw;
    if constexpr (!FLAT) smem += (128u - (smem_addr(smem_raw) & 127u)) & 127u;
    constexpr int G = 32 / LPS;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane / LPS, gl = lane % LPS;
    unsigned char *slot = smem + (size_t)(warp * G + g) * sbytes;
    float4 *pts = reinterpret_cast<float4 *>(slot);
    float *fr = reinterpret_cast<float *>(slot + 16 * W.max_points);
    float *th = fr + 12 * W.max_links;
    float *th_old = th + W.max_links;
    float4 *tb = reinterpret_cast<float4 *>(slot + tiles_offset(W.max_points, W.max_links));
    // (arenas) the scene's exchange area, after all slots of the block
    unsigned char *xch = smem + (size_t)(blockDim.x / 32) * G * sbytes + (size_t)(warp * G + g) * xch_bytes(W.max_chunks);
    const long long step0 = *W.step;
    const int n_sched = W.sched_count ? *W.sched_count : W.n_sched;
    const int n_items = (n_sched + G - 1) / G;
    for (;;) {
        int item = 0;
        if (lane == 0) item = (int)atomicAdd(W.queue, 1u);
        item = __shfl_sync(FULL_MASK, item, 0);
        if (item >= n_items) break;
        const int idx = item * G + g;
        const int s = idx < n_sched ? W.order[idx] : -1;
        run_scene<LPS, FLAT, OPT, ARENA>(W, s, gl, pts, fr, th, th_old, tb, n_steps, step0, xch, sbytes, tmap, item);
    }
}

// Flat ground: up to 16 warps per block, 128 registers a thread.
template <int LPS, bool OPT>
__global__ void __launch_bounds__(512) step_kernel(const __grid_constant__ WorldDev W, int n_steps, int sbytes,
                                                   const __grid_constant__ CUtensorMap tmap) {
    step_body<LPS, true, OPT, false>(W, n_steps, sbytes, &tmap);
}

// Height maps keep more state (the map window and its origin): 168 registers a thread, up to 12
// warps per block; their larger slots leave no more warps resident at 16 lanes per scene anyway.
template <int LPS, bool OPT>
__global__ void __maxnreg__(168) step_kernel_hm(const __grid_constant__ WorldDev W, int n_steps, int sbytes,
                                                const __grid_constant__ CUtensorMap tmap) {
    step_body<LPS, false, OPT, false>(W, n_steps, sbytes, &tmap);
}

// Arenas (robots colliding with one another, 8 or 16 lanes per scene), with the friction options
// compiled in: 168 registers a thread.
template <int LPS, bool FLAT>
__global__ void __maxnreg__(168) step_kernel_arena(const __grid_constant__ WorldDev W, int n_steps, int sbytes,
                                                   const __grid_constant__ CUtensorMap tmap) {
    step_body<LPS, FLAT, true, true>(W, n_steps, sbytes, &tmap);
}

__global__ void advance_kernel(long long *step, int n) { *step += n; }

// ------------------------------------------------------------------------ state set-up and probes

// One warp per scene: joint angles already in W.theta; origin/quat/vel/omega are the caller's
// arrays (AoS, [S*3] / [S*4]).  CoG = origin + R g, L = R Ib R^T omega, contact history cleared.
__global__ void __launch_bounds__(128) init_kernel(const __grid_constant__ WorldDev W, const float *origin, const float *quat,
                                                   const float *vel, const float *omega, int sbytes) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int s = blockIdx.x * (blockDim.x >> 5) + warp;
    if (s >= W.S) return;   // warp-uniform
    unsigned char *slot = smem + (size_t)warp * sbytes;
    float4 *pts = reinterpret_cast<float4 *>(slot);
    float *fr = reinterpret_cast<float *>(slot + 16 * W.max_points);
    float *th = fr + 12 * W.max_links;
    const int p0 = W.point_off[s], np = W.point_off[s + 1] - p0;
    const int l0 = W.link_off[s], nl = W.link_off[s + 1] - l0, j0 = l0 - s;
    for (int j = lane; j < nl - 1; j += 32) th[j] = W.theta[j0 + j];
    __syncwarp();
    Shape sh;
    shape_update<32>(W, s, p0, np, l0, nl, th, fr, pts, lane, sh);
    for (int i = lane; i < np; i += 32) W.kappa[p0 + i] = 0;
    if (lane == 0) {
        float q[4] = {quat[4 * s], quat[4 * s + 1], quat[4 * s + 2], quat[4 * s + 3]};
        const float inv = 1.0f / sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        q[0] *= inv; q[1] *= inv; q[2] *= inv; q[3] *= inv;
        float R[9], Rg[3], L[3];
        quat_mat(q, R);
        mat_vec(R, sh.g, Rg);
        const float w[3] = {omega[3 * s], omega[3 * s + 1], omega[3 * s + 2]};
        world_sym(R, sh.Ib, w, L);
        const int S = W.S;
        W.st[ST_CX * S + s] = origin[3 * s] + Rg[0];
        W.st[ST_CY * S + s] = origin[3 * s + 1] + Rg[1];
        W.st[ST_CZ * S + s] = origin[3 * s + 2] + Rg[2];
        W.st[ST_QW * S + s] = q[0]; W.st[ST_QX * S + s] = q[1];
        W.st[ST_QY * S + s] = q[2]; W.st[ST_QZ * S + s] = q[3];
        W.st[ST_VX * S + s] = vel[3 * s]; W.st[ST_VY * S + s] = vel[3 * s + 1];
        W.st[ST_VZ * S + s] = vel[3 * s + 2];
        W.st[ST_LX * S + s] = L[0]; W.st[ST_LY * S + s] = L[1]; W.st[ST_LZ * S + s] = L[2];
        W.omega[s] = w[0]; W.omega[S + s] = w[1]; W.omega[2 * S + s] = w[2];
        W.sensors[s] = 0u;
        W.status[s] = 0u;
    }
}

// Angular velocity of every scene from its state (one warp per scene), after a raw state write.
__global__ void __launch_bounds__(128) refresh_kernel(const __grid_constant__ WorldDev W, int sbytes) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int s = blockIdx.x * (blockDim.x >> 5) + warp;
    if (s >= W.S) return;   // warp-uniform
    unsigned char *slot = smem + (size_t)warp * sbytes;
    float4 *pts = reinterpret_cast<float4 *>(slot);
    float *fr = reinterpret_cast<float *>(slot + 16 * W.max_points);
    float *th = fr + 12 * W.max_links;
    const int p0 = W.point_off[s], np = W.point_off[s + 1] - p0;
    const int l0 = W.link_off[s], nl = W.link_off[s + 1] - l0, j0 = l0 - s;
    for (int j = lane; j < nl - 1; j += 32) th[j] = W.theta[j0 + j];
    __syncwarp();
    Shape sh;
    shape_update<32>(W, s, p0, np, l0, nl, th, fr, pts, lane, sh);
    uint32_t sens = 0;   // contact sensors of the written contact flags
    for (int i = lane; i < np; i += 32) {
        if (!W.kappa[p0 + i]) continue;
        const int sid = W.links[l0 + W.plink[p0 + i]].sensor;
        if (sid >= 0 && sid < 32) sens |= 1u << sid;
    }
    sens = gor<32>(sens);
    if (lane == 0) {
        const int S = W.S;
        const float q[4] = {W.st[ST_QW * S + s], W.st[ST_QX * S + s], W.st[ST_QY * S + s],
                            W.st[ST_QZ * S + s]};
        const float L[3] = {W.st[ST_LX * S + s], W.st[ST_LY * S + s], W.st[ST_LZ * S + s]};
        float R[9], om[3];
        quat_mat(q, R);
        world_sym(R, sh.Ii, L, om);
        W.omega[s] = om[0]; W.omega[S + s] = om[1]; W.omega[2 * S + s] = om[2];
        W.sensors[s] = sens;
    }
}

// World positions x_i = c + R r_i of one scene's points (one warp).
__global__ void __launch_bounds__(32) points_kernel(const __grid_constant__ WorldDev W, int s, float *out, int sbytes) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x;
    float4 *pts = reinterpret_cast<float4 *>(smem);
    float *fr = reinterpret_cast<float *>(smem + 16 * W.max_points);
    float *th = fr + 12 * W.max_links;
    const int p0 = W.point_off[s], np = W.point_off[s + 1] - p0;
    const int l0 = W.link_off[s], nl = W.link_off[s + 1] - l0, j0 = l0 - s;
    for (int j = lane; j < nl - 1; j += 32) th[j] = W.theta[j0 + j];
    __syncwarp();
    Shape sh;
    shape_update<32>(W, s, p0, np, l0, nl, th, fr, pts, lane, sh);
    const int S = W.S;
    const float c[3] = {W.st[ST_CX * S + s], W.st[ST_CY * S + s], W.st[ST_CZ * S + s]};
    const float q[4] = {W.st[ST_QW * S + s], W.st[ST_QX * S + s], W.st[ST_QY * S + s],
                        W.st[ST_QZ * S + s]};
    float R[9];
    quat_mat(q, R);
    for (int i = lane; i < np; i += 32) {
        const float4 r = pts[i];
        const float rr[3] = {r.x, r.y, r.z};
        float x[3];
        mat_vec(R, rr, x);
        out[3 * i] = c[0] + x[0]; out[3 * i + 1] = c[1] + x[1]; out[3 * i + 2] = c[2] + x[2];
    }
}

// ------------------------------------------------------------------------ learned surrogate
// The surrogate sees a scene through per-link features: per link, the CoG of its points
// (horizontally relative to a reference, z absolute), its orientation, the velocity of its CoG
// and the angular velocity (13 numbers; the robot is one rigid body, so every link shares it),
// then the joint angles after this step's joint update and the contact-sensor bits of the last
// step.  The link part is a function of the root state and the posed shape; the shape depends on
// the joint angles only, which change on joint-update steps (always taken by the plain step), so
// it is computed once per change into a per-scene cache (shape_cache_kernel) and the per-step
// kernels do no forward kinematics.

__device__ __forceinline__ Sym cached_sym(const float *a, int S, int s) {
    return Sym{a[0 * S + s], a[1 * S + s], a[2 * S + s], a[3 * S + s], a[4 * S + s], a[5 * S + s]};
}

struct RootState {
    float c[3], q[4], v[3], L[3];
};

__device__ __forceinline__ RootState load_root(const WorldDev &W, int s) {
    const int S = W.S;
    RootState r;
    r.c[0] = W.st[ST_CX * S + s]; r.c[1] = W.st[ST_CY * S + s]; r.c[2] = W.st[ST_CZ * S + s];
    r.q[0] = W.st[ST_QW * S + s]; r.q[1] = W.st[ST_QX * S + s]; r.q[2] = W.st[ST_QY * S + s];
    r.q[3] = W.st[ST_QZ * S + s];
    r.v[0] = W.st[ST_VX * S + s]; r.v[1] = W.st[ST_VY * S + s]; r.v[2] = W.st[ST_VZ * S + s];
    r.L[0] = W.st[ST_LX * S + s]; r.L[1] = W.st[ST_LY * S + s]; r.L[2] = W.st[ST_LZ * S + s];
    return r;
}

// The 13 features of one link: lq = link orientation in the body frame, lp = link CoG offset from
// the robot CoG in the body frame; R = root rotation, om = angular velocity.
__device__ __forceinline__ void link_features(const RootState &x, const float R[9], const float om[3],
                                              float4 lq, float4 lp, float rx, float ry, float f[13]) {
    const float ps[3] = {lp.x, lp.y, lp.z};
    const float ql[4] = {lq.x, lq.y, lq.z, lq.w};
    float r[3], qq[4];
    mat_vec(R, ps, r);
    quat_mul(x.q, ql, qq);
    f[0] = x.c[0] + r[0] - rx; f[1] = x.c[1] + r[1] - ry; f[2] = x.c[2] + r[2];
    f[3] = qq[0]; f[4] = qq[1]; f[5] = qq[2]; f[6] = qq[3];
    f[7] = x.v[0] + om[1] * r[2] - om[2] * r[1];
    f[8] = x.v[1] + om[2] * r[0] - om[0] * r[2];
    f[9] = x.v[2] + om[0] * r[1] - om[1] * r[0];
    f[10] = om[0]; f[11] = om[1]; f[12] = om[2];
}

// Number of points on contact-sensor links, per scene, and the largest (one warp per scene).
__global__ void __launch_bounds__(128) sensor_points_kernel(const __grid_constant__ WorldDev W, int *count, int *max_count) {
    const int lane = threadIdx.x & 31;
    const int s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (s >= W.S) return;   // warp-uniform
    const int p0 = W.point_off[s], np = W.point_off[s + 1] - p0, l0 = W.link_off[s];
    int c = 0;
    for (int i = lane; i < np; i += 32) {
        const int sid = W.links[l0 + W.plink[p0 + i]].sensor;
        c += (sid >= 0 && sid < 32) ? 1 : 0;
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(FULL_MASK, c, o);
    if (lane == 0) {
        count[s] = c;
        atomicMax(max_count, c);
    }
}

// The posed shape of every scene at its current joint angles, into the cache (one warp per scene).
__global__ void __launch_bounds__(128) shape_cache_kernel(const __grid_constant__ WorldDev W, SurCache C, int sbytes) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int s = blockIdx.x * (blockDim.x >> 5) + warp;
    if (s >= W.S) return;   // warp-uniform
    unsigned char *slot = smem + (size_t)warp * sbytes;
    float4 *pts = reinterpret_cast<float4 *>(slot);
    float *fr = reinterpret_cast<float *>(slot + 16 * W.max_points);
    float *th = fr + 12 * W.max_links;
    const int p0 = W.point_off[s], np = W.point_off[s + 1] - p0;
    const int l0 = W.link_off[s], nl = W.link_off[s + 1] - l0, j0 = l0 - s;
    for (int j = lane; j < nl - 1; j += 32) th[j] = W.theta[j0 + j];
    __syncwarp();
    Shape sh;
    shape_update<32>(W, s, p0, np, l0, nl, th, fr, pts, lane, sh);
    for (int l = lane; l < C.nl; l += 32) {
        float4 lq = make_float4(1.f, 0.f, 0.f, 0.f), lp = make_float4(0.f, 0.f, 0.f, 0.f);
        if (l < nl) {
            const float *F = fr + 12 * l;
            const float pc[3] = {W.link_cog[3 * (l0 + l)], W.link_cog[3 * (l0 + l) + 1], W.link_cog[3 * (l0 + l) + 2]};
            float ql[4];
            quat_from_mat(F, ql);
            lq = make_float4(ql[0], ql[1], ql[2], ql[3]);
            lp.x = F[0] * pc[0] + F[1] * pc[1] + F[2] * pc[2] + F[9] - sh.g[0];
            lp.y = F[3] * pc[0] + F[4] * pc[1] + F[5] * pc[2] + F[10] - sh.g[1];
            lp.z = F[6] * pc[0] + F[7] * pc[1] + F[8] * pc[2] + F[11] - sh.g[2];
        }
        C.lk[((size_t)s * C.nl + l) * 2] = lq;
        C.lk[((size_t)s * C.nl + l) * 2 + 1] = lp;
    }
    if (lane == 0) {
        const int S = W.S;
        const float v[12] = {sh.Ib.xx, sh.Ib.yy, sh.Ib.zz, sh.Ib.xy, sh.Ib.xz, sh.Ib.yz,
                             sh.Ii.xx, sh.Ii.yy, sh.Ii.zz, sh.Ii.xy, sh.Ii.xz, sh.Ii.yz};
        for (int k = 0; k < 12; ++k) C.inert[k * S + s] = v[k];
    }
    // the points of sensor links, compacted in stored order
    int base = 0;
    for (int i0 = 0; i0 < np; i0 += 32) {
        const int i = i0 + lane;
        int sid = -1;
        if (i < np) sid = W.links[l0 + W.plink[p0 + i]].sensor;
        const bool is = sid >= 0 && sid < 32;
        const unsigned m = __ballot_sync(FULL_MASK, is);
        if (is) {
            const int k = base + __popc(m & ((1u << lane) - 1u));
            const float4 r = pts[i];
            if (k < C.nsp) C.spt[(size_t)s * C.nsp + k] = make_float4(r.x, r.y, r.z, (float)sid);
        }
        base += __popc(m);
    }
}

// The same cache copied from the posed-shape cache when every scene's entry is current (its link
// entries were written with the shape): one warp per scene, no shape rebuilt.
__global__ void __launch_bounds__(256) shape_cache_copy_kernel(const __grid_constant__ WorldDev W, SurCache C) {
    const int lane = threadIdx.x & 31;
    const int s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (s >= W.S) return;   // warp-uniform
    const int nl = W.link_off[s + 1] - W.link_off[s];
    const float4 *e = W.scache + (size_t)s * scache_stride(W.scache_mp, W.scache_mt, W.scache_ml);
    const float4 *m = e + W.scache_mp + 2 * W.scache_mt;
    const float4 *lk = m + 5;
    for (int l = lane; l < C.nl; l += 32) {
        float4 lq = make_float4(1.f, 0.f, 0.f, 0.f), lp = make_float4(0.f, 0.f, 0.f, 0.f);
        if (l < nl) { lq = lk[2 * l]; lp = lk[2 * l + 1]; }
        C.lk[((size_t)s * C.nl + l) * 2] = lq;
        C.lk[((size_t)s * C.nl + l) * 2 + 1] = lp;
    }
    if (lane < 12) {
        const float4 m1 = m[1], m2 = m[2], m3 = m[3];
        const float v[12] = {m1.x, m1.y, m1.z, m1.w, m2.x, m2.y, m2.z, m2.w, m3.x, m3.y, m3.z, m3.w};
        float x = v[0];
#pragma unroll
        for (int k = 1; k < 12; ++k) x = lane == k ? v[k] : x;
        C.inert[lane * W.S + s] = x;
    }
    const int n = min(C.nsp_s[s], C.nsp);
    for (int k = lane; k < n; k += 32) {
        const int x = C.sidx[(size_t)s * C.nsp + k];
        const float4 r = e[x & 0xffff];
        C.spt[(size_t)s * C.nsp + k] = make_float4(r.x, r.y, r.z, (float)(x >> 16));
    }
}

// Each scene's sensor points in stored order: their index within the scene and sensor bit (one
// warp per scene; the order the shape caches write them in).
__global__ void __launch_bounds__(128) sensor_index_kernel(const __grid_constant__ WorldDev W, SurCache C) {
    const int lane = threadIdx.x & 31;
    const int s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (s >= W.S) return;   // warp-uniform
    const int p0 = W.point_off[s], np = W.point_off[s + 1] - p0, l0 = W.link_off[s];
    int base = 0;
    for (int i0 = 0; i0 < np; i0 += 32) {
        const int i = i0 + lane;
        int sid = -1;
        if (i < np) sid = W.links[l0 + W.plink[p0 + i]].sensor;
        const bool is = sid >= 0 && sid < 32;
        const unsigned msk = __ballot_sync(FULL_MASK, is);
        if (is) {
            const int k = base + __popc(msk & ((1u << lane) - 1u));
            if (k < C.nsp) C.sidx[(size_t)s * C.nsp + k] = i | (sid << 16);
        }
        base += __popc(msk);
    }
}

// Features of every scene, one thread per (scene, link): the link's 13 features, the angle of the
// joint that drives the link and the sensor bits k = link (mod links).  Outputs: FP32 (standardised
// when x_mu is set), raw, BF16 standardised into the network's input rows (whose padding columns
// are zero and are not written), and the delta target against the raw features of the previous
// state.
// per-scene values a features block computes once: CoG, orientation, velocity, angular velocity,
// rotation matrix, horizontal reference and sensor word
enum { FS_C = 0, FS_Q = 3, FS_V = 7, FS_W = 10, FS_R = 13, FS_RX = 22, FS_RY = 23, FS_SENS = 24, FS_N = 25 };

__global__ void __launch_bounds__(256) features_kernel(const __grid_constant__ WorldDev W, SurCache C, SurrogateIO io, int spb) {
    // [spb x nfp] raw features of the block's scenes (rows padded to whole float4), then
    // [spb x FS_N] per-scene values
    extern __shared__ __align__(16) float rows[];
    __shared__ int tick;
    const int tid = threadIdx.x, S = W.S, nfp = (io.nf + 3) & ~3;
    const int s0 = blockIdx.x * spb, ns = min(spb, S - s0);
    float *sv = rows + (size_t)spb * nfp;
    const long long n = *W.step;
    // every (scene, link) thread issues its loads first, so that they overlap the per-scene phase
    const bool mine = tid < ns * io.nl;
    const int sl = mine ? tid / io.nl : 0, l = mine ? tid % io.nl : 0, s = s0 + sl;
    int l0 = 0, nl = 0;
    float4 lq = make_float4(1.f, 0.f, 0.f, 0.f), lp = make_float4(0.f, 0.f, 0.f, 0.f);
    float th = 0.f;
    if (mine) {
        l0 = W.link_off[s];
        nl = W.link_off[s + 1] - l0;
        if (l < nl) {
            lq = C.lk[((size_t)s * C.nl + l) * 2];
            lp = C.lk[((size_t)s * C.nl + l) * 2 + 1];
        }
        if (l >= 1 && l - 1 < nl - 1) th = W.theta[l0 - s + l - 1];
    }
    if (tid < ns) {   // one thread per scene: the scene's rotation and angular velocity
        const int s = s0 + tid;
        const RootState x = load_root(W, s);
        float R[9], om[3];
        quat_mat(x.q, R);
        world_sym(R, cached_sym(C.inert + 6 * S, S, s), x.L, om);
        float *p = sv + (size_t)tid * FS_N;
#pragma unroll
        for (int k = 0; k < 3; ++k) { p[FS_C + k] = x.c[k]; p[FS_V + k] = x.v[k]; p[FS_W + k] = om[k]; }
#pragma unroll
        for (int k = 0; k < 4; ++k) p[FS_Q + k] = x.q[k];
#pragma unroll
        for (int k = 0; k < 9; ++k) p[FS_R + k] = R[k];
        p[FS_RX] = io.cxy_ref ? io.cxy_ref[2 * s] : x.c[0];
        p[FS_RY] = io.cxy_ref ? io.cxy_ref[2 * s + 1] : x.c[1];
        p[FS_SENS] = __uint_as_float(W.sensors[s]);
        if (io.cxy_out) { io.cxy_out[2 * s] = x.c[0]; io.cxy_out[2 * s + 1] = x.c[1]; }
    }
    if (tid == 0) tick = W.act_mode != 0 && n % W.K == 0;   // the step's joint update (all scenes)
    __syncthreads();
    if (mine) {   // one thread per (scene, link)
        float *row = rows + (size_t)sl * nfp;
        const float *p = sv + (size_t)sl * FS_N;
        RootState x;
        float R[9], om[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) { x.c[k] = p[FS_C + k]; x.v[k] = p[FS_V + k]; om[k] = p[FS_W + k]; x.L[k] = 0.f; }
#pragma unroll
        for (int k = 0; k < 4; ++k) x.q[k] = p[FS_Q + k];
#pragma unroll
        for (int k = 0; k < 9; ++k) R[k] = p[FS_R + k];
        const int j0 = l0 - s;
        float f[13];
        if (l < nl) {
            link_features(x, R, om, lq, lp, p[FS_RX], p[FS_RY], f);
        } else {
#pragma unroll
            for (int k = 0; k < 13; ++k) f[k] = 0.f;
        }
#pragma unroll
        for (int k = 0; k < 13; ++k) row[13 * l + k] = f[k];
        if (l >= 1) {   // joint l - 1 drives link l: its angle after this step's joint update
            const int j = l - 1;
            float a = 0.f;
            if (j < nl - 1) {
                if (tick) {
                    const LinkDev lk = W.links[l0 + j + 1];
                    a = fminf(fmaxf(joint_target(W, j0 + j, n), lk.lo), lk.hi);
                } else {
                    a = th;
                }
            }
            row[13 * io.nl + j] = a;
        }
        const uint32_t sens = __float_as_uint(p[FS_SENS]);
        for (int k = l; k < io.ns; k += io.nl) row[14 * io.nl - 1 + k] = (float)((sens >> k) & 1u);
    }
    __syncthreads();
    // the block's rows are contiguous in every output: write them out in full lines
    if (io.X || io.Xraw || io.T) {
        for (int e = tid; e < ns * io.nf; e += blockDim.x) {
            const int sl = e / io.nf, col = e - sl * io.nf, s = s0 + sl;
            const float raw = rows[(size_t)sl * nfp + col];
            const size_t o = (size_t)s * io.nf + col;
            if (io.Xraw) io.Xraw[o] = raw;
            if (io.X) io.X[o] = io.x_mu ? (raw - io.x_mu[col]) * io.x_isd[col] : raw;
            if (io.T && col < io.nt) {
                const float d = raw - io.prev[o];
                io.T[(size_t)s * io.nt + col] = io.t_mu ? (d - io.t_mu[col]) / io.t_sd[col] : d;
            }
        }
    }
    if (io.Xb) {   // 8 BF16 (16 bytes) per store; the columns past nf are padding and stay zero
        // chunks wholly inside the row take whole float4 loads when the norms are 16-byte aligned
        // (the caller's arrays; the rows are padded to float4)
        const bool vec = ((reinterpret_cast<uintptr_t>(io.x_mu) | reinterpret_cast<uintptr_t>(io.x_isd)) & 15u) == 0;
        const int chunks = (io.nf + 7) >> 3, full = vec ? io.nf >> 3 : 0;
        for (int e = tid; e < ns * chunks; e += blockDim.x) {
            const int sl = e / chunks, ch = e - sl * chunks, c0 = ch * 8;
            float v[8];
            if (ch < full) {
                const float4 *r4 = reinterpret_cast<const float4 *>(rows + (size_t)sl * nfp + c0);
                const float4 ra = r4[0], rb = r4[1];
                v[0] = ra.x; v[1] = ra.y; v[2] = ra.z; v[3] = ra.w; v[4] = rb.x; v[5] = rb.y; v[6] = rb.z; v[7] = rb.w;
                if (io.x_mu) {
                    const float4 *m4 = reinterpret_cast<const float4 *>(io.x_mu + c0);
                    const float4 *i4 = reinterpret_cast<const float4 *>(io.x_isd + c0);
                    const float4 ma = __ldg(m4), mb = __ldg(m4 + 1), ia = __ldg(i4), ib = __ldg(i4 + 1);
                    const float mu[8] = {ma.x, ma.y, ma.z, ma.w, mb.x, mb.y, mb.z, mb.w};
                    const float is[8] = {ia.x, ia.y, ia.z, ia.w, ib.x, ib.y, ib.z, ib.w};
#pragma unroll
                    for (int k = 0; k < 8; ++k) v[k] = (v[k] - mu[k]) * is[k];
                }
            } else {   // the row's last, partial chunk (or unaligned norms)
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int col = c0 + k;
                    const float raw = col < io.nf ? rows[(size_t)sl * nfp + col] : 0.f;
                    v[k] = col < io.nf && io.x_mu ? (raw - io.x_mu[col]) * io.x_isd[col] : raw;
                }
            }
            uint32_t w[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const __nv_bfloat162 hv = __floats2bfloat162_rn(v[2 * k], v[2 * k + 1]);
                w[k] = *reinterpret_cast<const uint32_t *>(&hv);
            }
            *reinterpret_cast<uint4 *>(reinterpret_cast<__nv_bfloat16 *>(io.Xb) + (size_t)(s0 + sl) * io.ldb + c0) =
                make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

// Surrogate update, one thread per scene: the root state from the torso's predicted next state
// (position, orientation, CoG velocity, angular velocity) into the candidate buffer nx
// [NX_N * S]; applied[s] says whether scene s has a candidate (frozen scenes and non-finite
// predictions have none; the latter freeze the scene).
enum { NX_CX = 0, NX_CY, NX_CZ, NX_QW, NX_QX, NX_QY, NX_QZ, NX_VX, NX_VY, NX_VZ, NX_LX, NX_LY, NX_LZ,
       NX_WX, NX_WY, NX_WZ, NX_N };

__global__ void __launch_bounds__(256) surrogate_apply_kernel(const __grid_constant__ WorldDev W, SurCache C, const float *Y, int ldy,
                                                              const float *t_mu, const float *t_sd, float *nx,
                                                              uint8_t *applied) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= W.S) return;
    const int S = W.S;
    const uint32_t status = W.status[s];
    if (status) { applied[s] = 0; return; }
    const RootState x = load_root(W, s);
    float R[9], om[3];
    quat_mat(x.q, R);
    world_sym(R, cached_sym(C.inert + 6 * S, S, s), x.L, om);
    const float4 lq = C.lk[(size_t)s * C.nl * 2], lp = C.lk[(size_t)s * C.nl * 2 + 1];
    float f[13];
    link_features(x, R, om, lq, lp, x.c[0], x.c[1], f);
    const float *y = Y + (size_t)s * ldy;
#pragma unroll
    for (int i = 0; i < 13; ++i) f[i] += y[i] * t_sd[i] + t_mu[i];
    // torso orientation -> root orientation (the torso frame relative to the body frame is lq)
    float qt[4] = {f[3], f[4], f[5], f[6]};
    const float inv = rsqrtf(qt[0] * qt[0] + qt[1] * qt[1] + qt[2] * qt[2] + qt[3] * qt[3]);
    qt[0] *= inv; qt[1] *= inv; qt[2] *= inv; qt[3] *= inv;
    const float lqc[4] = {lq.x, -lq.y, -lq.z, -lq.w};
    float qn[4], Rn[9];
    quat_mul(qt, lqc, qn);
    quat_mat(qn, Rn);
    const float ps[3] = {lp.x, lp.y, lp.z};
    float d[3], L[3];
    mat_vec(Rn, ps, d);
    const float w[3] = {f[10], f[11], f[12]};
    const float c[3] = {x.c[0] + f[0] - d[0], x.c[1] + f[1] - d[1], f[2] - d[2]};
    const float v[3] = {f[7] - (w[1] * d[2] - w[2] * d[1]), f[8] - (w[2] * d[0] - w[0] * d[2]),
                        f[9] - (w[0] * d[1] - w[1] * d[0])};
    world_sym(Rn, cached_sym(C.inert, S, s), w, L);
    const float chk = c[0] + c[1] + c[2] + v[0] + v[1] + v[2] + L[0] + L[1] + L[2] + qn[0] + qn[1] + qn[2] + qn[3];
    if (!isfinite(chk)) {
        W.status[s] = status | 1u;
        applied[s] = 0;
        return;
    }
    const float o[NX_N] = {c[0], c[1], c[2], qn[0], qn[1], qn[2], qn[3], v[0], v[1], v[2], L[0], L[1], L[2],
                           w[0], w[1], w[2]};
#pragma unroll
    for (int k = 0; k < NX_N; ++k) nx[(size_t)k * S + s] = o[k];
    applied[s] = 1;
}

// Contact sensors at the candidate state, one warp per scene over its sensor points (the cached
// body-frame offsets of the points of contact-sensor links).
template <bool FLAT>
__global__ void __launch_bounds__(256) sensor_probe_kernel(const __grid_constant__ WorldDev W, SurCache C, const float *nx,
                                                           const uint8_t *applied, uint32_t *sens_new) {
    const int lane = threadIdx.x & 31;
    const int s = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (s >= W.S || !applied[s]) return;   // warp-uniform
    const int S = W.S;
    const float q[4] = {nx[NX_QW * S + s], nx[NX_QX * S + s], nx[NX_QY * S + s], nx[NX_QZ * S + s]};
    const float c[3] = {nx[NX_CX * S + s], nx[NX_CY * S + s], nx[NX_CZ * S + s]};
    const int n = C.nsp_s[s], hm = FLAT ? -1 : W.hmap[s];
    float R[9];
    quat_mat(q, R);
    uint32_t bits = 0u;
    for (int k = lane; k < n; k += 32) {
        const float4 r = C.spt[(size_t)s * C.nsp + k];
        const float px = c[0] + R[0] * r.x + R[1] * r.y + R[2] * r.z;
        const float py = c[1] + R[3] * r.x + R[4] * r.y + R[5] * r.z;
        const float pz = c[2] + R[6] * r.x + R[7] * r.y + R[8] * r.z;
        if (pz < ground<FLAT>(W, hm, px, py)) bits |= 1u << (int)r.w;
    }
    bits = gor<32>(bits);
    if (lane == 0) sens_new[s] = bits;
}

// One thread per scene: keep the candidate state if the contact sensors did not change, otherwise
// leave the scene at its state and append it to the fallback list (the plain step takes it).
__global__ void __launch_bounds__(256) surrogate_commit_kernel(const __grid_constant__ WorldDev W, const float *nx, const uint8_t *applied,
                                                               const uint32_t *sens_new, int *list, int *count, int *fb,
                                                               int max_changed) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const bool app = s < W.S && applied[s];
    const uint32_t sn = app ? sens_new[s] : 0u, so = app ? W.sensors[s] : 0u;
    const bool fall = app && __popc(sn ^ so) > max_changed;
    // warp-aggregated append
    const unsigned m = __ballot_sync(FULL_MASK, fall);
    int base = 0;
    const int lane = threadIdx.x & 31;
    if (m) {
        if (lane == __ffs(m) - 1) base = atomicAdd(count, __popc(m));
        base = __shfl_sync(FULL_MASK, base, __ffs(m) - 1);
    }
    if (fall) {
        list[base + __popc(m & ((1u << lane) - 1u))] = s;
        fb[s] += 1;   // one thread per scene
    }
    if (!app || fall) return;
    const int S = W.S;
    if (sn != so) W.sensors[s] = sn;   // a change the rule lets through
#pragma unroll
    for (int k = 0; k < ST_N; ++k) W.st[(size_t)k * S + s] = nx[(size_t)k * S + s];
    W.omega[s] = nx[NX_WX * S + s];
    W.omega[S + s] = nx[NX_WY * S + s];
    W.omega[2 * S + s] = nx[NX_WZ * S + s];
}

// Contact flags of every point and the contact sensors at the current state, for the listed scenes
// (list NULL: every scene) -- the previous-step contacts a plain step needs after surrogate steps.
template <bool FLAT>
__global__ void __launch_bounds__(128) kappa_refresh_kernel(const __grid_constant__ WorldDev W, const int *list, const int *count,
                                                            int sbytes) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    unsigned char *slot = smem + (size_t)warp * sbytes;
    float4 *pts = reinterpret_cast<float4 *>(slot);
    float *fr = reinterpret_cast<float *>(slot + 16 * W.max_points);
    float *th = fr + 12 * W.max_links;
    const int n = list ? *count : W.S;
    for (int i = blockIdx.x * wpb + warp; i < n; i += gridDim.x * wpb) {   // warp-uniform
        const int s = list ? list[i] : i;
        const int p0 = W.point_off[s], np = W.point_off[s + 1] - p0;
        const int l0 = W.link_off[s], nl = W.link_off[s + 1] - l0, j0 = l0 - s;
        for (int j = lane; j < nl - 1; j += 32) th[j] = W.theta[j0 + j];
        __syncwarp();
        Shape sh;
        shape_update<32>(W, s, p0, np, l0, nl, th, fr, pts, lane, sh);
        const RootState x = load_root(W, s);
        float R[9];
        quat_mat(x.q, R);
        const int hm = FLAT ? -1 : W.hmap[s];
        uint32_t sens = 0;
        for (int k = lane; k < np; k += 32) {
            const float4 r = pts[k];
            const float px = x.c[0] + R[0] * r.x + R[1] * r.y + R[2] * r.z;
            const float py = x.c[1] + R[3] * r.x + R[4] * r.y + R[5] * r.z;
            const float pz = x.c[2] + R[6] * r.x + R[7] * r.y + R[8] * r.z;
            const bool kap = pz < ground<FLAT>(W, hm, px, py);
            W.kappa[p0 + k] = kap ? 1 : 0;
            if (kap) {
                const int sid = W.links[l0 + W.plink[p0 + k]].sensor;
                if (sid >= 0 && sid < 32) sens |= 1u << sid;
            }
        }
        sens = gor<32>(sens);
        if (lane == 0) W.sensors[s] = sens;
        __syncwarp();
    }
}

__global__ void accumulate_kernel(long long *total, int *count, int mult) {
    *total += (long long)*count * mult;
    *count = 0;
}

cudaError_t launch_accumulate(long long *total, int *count, int mult, cudaStream_t st) {
    accumulate_kernel<<<1, 1, 0, st>>>(total, count, mult);
    return cudaGetLastError();
}

namespace {
constexpr int SUR_WPB = 4;   // warps (scenes) per block of the surrogate kernels
unsigned sur_blocks(int S) { return (unsigned)((S + SUR_WPB - 1) / SUR_WPB); }
}  // namespace

cudaError_t launch_sensor_points(const WorldDev &W, int *count, int *max_count, cudaStream_t st) {
    sensor_points_kernel<<<sur_blocks(W.S), SUR_WPB * 32, 0, st>>>(W, count, max_count);
    return cudaGetLastError();
}

cudaError_t launch_sensor_index(const WorldDev &W, const SurCache &C, cudaStream_t st) {
    sensor_index_kernel<<<sur_blocks(W.S), SUR_WPB * 32, 0, st>>>(W, C);
    return cudaGetLastError();
}

cudaError_t launch_shape_cache(const WorldDev &W, const SurCache &C, cudaStream_t st) {
    if (W.scache_mode == 2) {   // every scene's posed-shape entry is current: copy it
        shape_cache_copy_kernel<<<(unsigned)((W.S + 7) / 8), 256, 0, st>>>(W, C);
        return cudaGetLastError();
    }
    const int sb = (int)slot_bytes(W.max_points, W.max_links, 32);
    cudaError_t e = cudaFuncSetAttribute((void *)shape_cache_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         SUR_WPB * sb);
    if (e != cudaSuccess) return e;
    shape_cache_kernel<<<sur_blocks(W.S), SUR_WPB * 32, SUR_WPB * sb, st>>>(W, C, sb);
    return cudaGetLastError();
}

cudaError_t launch_features(const WorldDev &W, const SurCache &C, const SurrogateIO &io, cudaStream_t st) {
    const int spb = io.nl >= 256 ? 1 : 256 / io.nl;             // scenes per block
    const int threads = std::max(256, (io.nl + 31) / 32 * 32);
    const size_t sm = (size_t)spb * (((io.nf + 3) & ~3) + FS_N) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute((void *)features_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    features_kernel<<<(unsigned)((W.S + spb - 1) / spb), threads, sm, st>>>(W, C, io, spb);
    return cudaGetLastError();
}

cudaError_t launch_surrogate_update(const WorldDev &W, const SurCache &C, const float *Y, int ldy, const float *t_mu,
                                    const float *t_sd, float *nx, uint8_t *applied, uint32_t *sens_new, int *list,
                                    int *count, int *fb, int max_changed, cudaStream_t st) {
    const unsigned bs = (unsigned)((W.S + 255) / 256);
    surrogate_apply_kernel<<<bs, 256, 0, st>>>(W, C, Y, ldy, t_mu, t_sd, nx, applied);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const unsigned bp = (unsigned)(((long long)W.S * 32 + 255) / 256);
    if (W.hm)
        sensor_probe_kernel<false><<<bp, 256, 0, st>>>(W, C, nx, applied, sens_new);
    else
        sensor_probe_kernel<true><<<bp, 256, 0, st>>>(W, C, nx, applied, sens_new);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    surrogate_commit_kernel<<<bs, 256, 0, st>>>(W, nx, applied, sens_new, list, count, fb, max_changed);
    return cudaGetLastError();
}

cudaError_t launch_kappa_refresh(const WorldDev &W, const int *list, const int *count, cudaStream_t st) {
    const int sb = (int)slot_bytes(W.max_points, W.max_links, 32);
    void *fn = W.hm ? (void *)kappa_refresh_kernel<false> : (void *)kappa_refresh_kernel<true>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, SUR_WPB * sb);
    if (e != cudaSuccess) return e;
    // a grid-stride loop over the scenes (or the listed ones), at most a few blocks per SM
    int dev = 0, nsm = 1;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const unsigned blocks = std::min(sur_blocks(W.S), (unsigned)(8 * nsm));
    WorldDev w = W;
    const int *l = list, *c = count;
    int sbv = sb;
    void *args[] = {&w, &l, &c, &sbv};
    return cudaLaunchKernel(fn, dim3(blocks), dim3(SUR_WPB * 32), args, SUR_WPB * sb, st);
}

// ------------------------------------------------------------------------ state in and out
// The caller's arrays are per scene (AoS: cog[3S], quat[4S], vel[3S], angmom[3S], omega[3S]) and its
// points in its own order; the device keeps SoA state and points by construction height (perm[i] =
// the caller's index of stored point i).  These kernels do the transposes and permutations next to
// the data, so a state exchange is one copy each way.

// staged AoS state (cog | quat | vel | angmom blocks) -> SoA state
__global__ void scatter_state_kernel(WorldDev W, const float *aos) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= W.S) return;
    const int S = W.S;
    const float *cog = aos, *quat = aos + 3 * S, *vel = aos + 7 * S, *L = aos + 10 * S;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        W.st[(ST_CX + k) * S + s] = cog[3 * s + k];
        W.st[(ST_VX + k) * S + s] = vel[3 * s + k];
        W.st[(ST_LX + k) * S + s] = L[3 * s + k];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) W.st[(ST_QW + k) * S + s] = quat[4 * s + k];
}

// SoA state and angular velocity -> AoS blocks cog | quat | vel | omega | angmom
__global__ void gather_state_kernel(WorldDev W, float *aos) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= W.S) return;
    const int S = W.S;
    float *cog = aos, *quat = aos + 3 * S, *vel = aos + 7 * S, *om = aos + 10 * S, *L = aos + 13 * S;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        cog[3 * s + k] = W.st[(ST_CX + k) * S + s];
        vel[3 * s + k] = W.st[(ST_VX + k) * S + s];
        om[3 * s + k] = W.omega[k * S + s];
        L[3 * s + k] = W.st[(ST_LX + k) * S + s];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) quat[4 * s + k] = W.st[(ST_QW + k) * S + s];
}

// contact flags: caller order -> stored order (to_stored) or back
__global__ void permute_kappa_kernel(uint8_t *dst, const uint8_t *src, const int *perm, int P, int to_stored) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    if (to_stored) dst[i] = src[perm[i]] ? 1 : 0;
    else dst[perm[i]] = src[i];
}

cudaError_t launch_scatter_state(const WorldDev &W, const float *aos, cudaStream_t st) {
    scatter_state_kernel<<<(W.S + 255) / 256, 256, 0, st>>>(W, aos);
    return cudaGetLastError();
}
cudaError_t launch_gather_state(const WorldDev &W, float *aos, cudaStream_t st) {
    gather_state_kernel<<<(W.S + 255) / 256, 256, 0, st>>>(W, aos);
    return cudaGetLastError();
}
cudaError_t launch_permute_kappa(uint8_t *dst, const uint8_t *src, const int *perm, int P, bool to_stored,
                                 cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    permute_kappa_kernel<<<(P + 255) / 256, 256, 0, st>>>(dst, src, perm, P, to_stored ? 1 : 0);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------ host-side launchers

// per-scene shared memory of the step kernel: the slot, plus the height-map window on maps
int step_slot_bytes(const WorldDev &W, int lps) {
    return W.hm ? hm_win_offset(W.max_points, W.max_links, lps) + HM_AREA : slot_bytes(W.max_points, W.max_links, lps);
}

size_t step_smem_bytes(const WorldDev &W, int lps, int wpb) {
    // (height maps) 128 more bytes to align the slots' windows for TMA
    return (size_t)wpb * (32 / lps) * (step_slot_bytes(W, lps) + (W.arena > 1 ? xch_bytes(W.max_chunks) : 0)) +
           (W.hm ? 128 : 0);
}

// One pass of the dilated height map: the highest cell within R cells along x (along_y = 0) or y
// (along_y = 1), clamped to the map; two passes give the maximum over the (2R + 1)^2 square.
__global__ void hm_dilate_kernel(const float *in, float *out, int H, int ny, int nx, int R, int along_y) {
    const size_t n = (size_t)H * ny * nx;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % (size_t)nx), y = (int)((i / (size_t)nx) % (size_t)ny);
        float m = -INFINITY;
        if (along_y) {
            const float *col = in + (i - (size_t)y * nx);
            for (int k = max(y - R, 0); k <= min(y + R, ny - 1); ++k) m = fmaxf(m, col[(size_t)k * nx]);
        } else {
            const float *row = in + (i - x);
            for (int k = max(x - R, 0); k <= min(x + R, nx - 1); ++k) m = fmaxf(m, row[k]);
        }
        out[i] = m;
    }
}

cudaError_t launch_hm_dilate(const float *hm, float *tmp, float *out, int H, int ny, int nx, int R,
                             cudaStream_t st) {
    const size_t n = (size_t)H * ny * nx;
    const int blocks = (int)std::min<size_t>((n + 255) / 256, 152 * 64);
    hm_dilate_kernel<<<blocks, 256, 0, st>>>(hm, tmp, H, ny, nx, R, 0);
    hm_dilate_kernel<<<blocks, 256, 0, st>>>(tmp, out, H, ny, nx, R, 1);
    return cudaGetLastError();
}

// The window wait on its own: one warp in groups of 8 lanes, each group with an mbarrier in shared
// memory; groups 0 and 2 arm theirs for a copy that is never issued (an arrival that expects
// HM_BOX x HM_WIN x 4 bytes), groups 1 and 3 complete theirs at once.  Every lane then waits with
// win_wait_warp.  out[0] = lanes whose wait gave up, out[1] = lanes that saw their barrier
// complete, out[2] = microseconds the wait took (lane 0).
__global__ void __launch_bounds__(32) window_wait_selftest_kernel(int *out) {
    __shared__ uint64_t bars[4];
    const int lane = threadIdx.x, g = lane / 8;
    if (lane % 8 == 0) win_bar_init(&bars[g]);
    __syncwarp();
    if (lane % 8 == 0) {
        if (g % 2 == 0)
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(&bars[g])),
                         "r"((uint32_t)(HM_BOX * HM_WIN * sizeof(float)))
                         : "memory");
        else
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&bars[g])) : "memory");
    }
    __syncwarp();
    unsigned long long t0, t1;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    const bool landed = win_wait_warp(&bars[g], 0u, true);
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
    const unsigned up = __ballot_sync(FULL_MASK, !landed), ok = __ballot_sync(FULL_MASK, landed);
    __syncwarp();
    if (lane % 8 == 0) win_bar_inval(&bars[g]);
    if (lane == 0) {
        out[0] = __popc(up);
        out[1] = __popc(ok);
        out[2] = (int)((t1 - t0) / 1000ull);
    }
}

typedef CUresult (*TmapEncodeFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

void encode_hm_tmap(WorldDev &W, int n_maps, CUtensorMap *out) {
    W.hm_tma = 0;
    W.hm_tmap_h = nullptr;
    if (!W.hm || n_maps < 1 || W.hm_nx < HM_WIN || W.hm_ny < HM_WIN || (W.hm_nx * 4) % 16 != 0 ||
        (reinterpret_cast<uintptr_t>(W.hm) & 15) != 0)
        return;
    static TmapEncodeFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return;
        fn = reinterpret_cast<TmapEncodeFn>(p);
    }
    const cuuint64_t dims[3] = {(cuuint64_t)W.hm_nx, (cuuint64_t)W.hm_ny, (cuuint64_t)n_maps};
    const cuuint64_t strides[2] = {(cuuint64_t)W.hm_nx * 4, (cuuint64_t)W.hm_nx * W.hm_ny * 4};
    const cuuint32_t box[3] = {HM_BOX, HM_WIN, 1};
    const cuuint32_t es[3] = {1, 1, 1};
    if (fn(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(W.hm), dims, strides, box, es,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS) {
        W.hm_tma = 1;
        W.hm_tmap_h = out;
    }
}

template <int LPS, bool FLAT, bool OPT>
static void *step_fn() { return FLAT ? (void *)step_kernel<LPS, OPT> : (void *)step_kernel_hm<LPS, OPT>; }

template <bool OPT>
static void *pick_step_opt(int lps, bool flat) {
    switch (lps) {
        case 4: return flat ? step_fn<4, true, OPT>() : step_fn<4, false, OPT>();
        case 8: return flat ? step_fn<8, true, OPT>() : step_fn<8, false, OPT>();
        case 16: return flat ? step_fn<16, true, OPT>() : step_fn<16, false, OPT>();
        case 32: return flat ? step_fn<32, true, OPT>() : step_fn<32, false, OPT>();
        default: return nullptr;
    }
}

// the kernel for a world: flat or height maps, friction options compiled in only when used,
// arenas (8 or 16 lanes per scene) in their own build
static void *pick_step(const WorldDev &W, int lps) {
    const bool flat = W.hm == nullptr;
    if (W.arena > 1) {
        if (lps == 8) return flat ? (void *)step_kernel_arena<8, true> : (void *)step_kernel_arena<8, false>;
        if (lps == 16) return flat ? (void *)step_kernel_arena<16, true> : (void *)step_kernel_arena<16, false>;
        return nullptr;
    }
    return W.fric_mode ? pick_step_opt<true>(lps, flat) : pick_step_opt<false>(lps, flat);
}

int step_blocks_per_sm(const WorldDev &W, int lps, int wpb, cudaError_t *err) {
    void *fn = pick_step(W, lps);
    *err = cudaSuccess;
    if (!fn) { *err = cudaErrorInvalidValue; return 0; }
    const size_t smem = step_smem_bytes(W, lps, wpb);
    // a shape over the per-block limit does not fit: report 0 blocks without a failing call (a
    // failed runtime call would leave an error behind for the next launch check to pick up)
    int dev = 0, optin = 0;
    if ((*err = cudaGetDevice(&dev)) != cudaSuccess) return 0;
    if ((*err = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return 0;
    if (smem > (size_t)optin) return 0;
    // the attribute is an upper limit: raise it, never lower it, so that a shape set up earlier
    // (another world, or the fallback shape of this one) stays launchable
    cudaFuncAttributes fa{};
    *err = cudaFuncGetAttributes(&fa, fn);
    if (*err != cudaSuccess) { cudaGetLastError(); return 0; }
    if (wpb * 32 > fa.maxThreadsPerBlock) return 0;
    if ((size_t)fa.maxDynamicSharedSizeBytes < smem) {
        *err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (*err != cudaSuccess) { cudaGetLastError(); return 0; }
    }
    int nb = 0;
    *err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, wpb * 32, smem);
    return nb;
}

cudaError_t launch_step(const WorldDev &W, const LaunchCfg &cfg, int n_steps, cudaStream_t st) {
    void *fn = pick_step(W, cfg.lps);
    if (!fn || cfg.wpb < 1 || cfg.wpb > 16 || cfg.blocks < 1) return cudaErrorInvalidValue;
    // the kernel's shared-memory limit was raised by step_blocks_per_sm for this shape
    const size_t smem = step_smem_bytes(W, cfg.lps, cfg.wpb);
    cudaError_t e = cudaMemsetAsync(W.queue, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    int sb = step_slot_bytes(W, cfg.lps);
    WorldDev w = W;
    CUtensorMap tm;
    if (W.hm_tma && W.hm_tmap_h) tm = *W.hm_tmap_h;
    else memset(&tm, 0, sizeof tm);
    void *args[] = {&w, &n_steps, &sb, &tm};
    return cudaLaunchKernel(fn, dim3(cfg.blocks), dim3(cfg.wpb * 32), args, smem, st);
}

cudaError_t launch_advance(long long *d_step, int n, cudaStream_t st) {
    advance_kernel<<<1, 1, 0, st>>>(d_step, n);
    return cudaGetLastError();
}

cudaError_t launch_init(const WorldDev &W, const float *d_origin, const float *d_quat,
                        const float *d_vel, const float *d_omega, cudaStream_t st) {
    const int wpb = 4;
    const int sb = slot_bytes(W.max_points, W.max_links, 32);
    const size_t smem = (size_t)wpb * sb;
    cudaError_t e = cudaFuncSetAttribute((void *)init_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    init_kernel<<<(W.S + wpb - 1) / wpb, wpb * 32, smem, st>>>(W, d_origin, d_quat, d_vel, d_omega, sb);
    return cudaGetLastError();
}

cudaError_t launch_refresh(const WorldDev &W, cudaStream_t st) {
    const int wpb = 4;
    const int sb = slot_bytes(W.max_points, W.max_links, 32);
    const size_t smem = (size_t)wpb * sb;
    cudaError_t e = cudaFuncSetAttribute((void *)refresh_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    refresh_kernel<<<(W.S + wpb - 1) / wpb, wpb * 32, smem, st>>>(W, sb);
    return cudaGetLastError();
}

cudaError_t launch_points(const WorldDev &W, int scene, float *d_out, cudaStream_t st) {
    const int sb = slot_bytes(W.max_points, W.max_links, 32);
    cudaError_t e = cudaFuncSetAttribute((void *)points_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, sb);
    if (e != cudaSuccess) return e;
    points_kernel<<<1, 32, sb, st>>>(W, scene, d_out, sb);
    return cudaGetLastError();
}

}  // namespace npx

extern "C" int npx_window_wait_selftest(int *gave_up, int *completed, int *elapsed_us, void *stream) {
    if (!gave_up || !completed || !elapsed_us)
        return npx::set_last_error(NPX_EINVAL, "npx_window_wait_selftest: null argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int *d = nullptr;
    cudaError_t e = cudaMalloc(&d, 3 * sizeof(int));
    if (e != cudaSuccess) return npx::set_last_error(NPX_ENOMEM, cudaGetErrorString(e));
    int h[3] = {-1, -1, -1};
    npx::window_wait_selftest_kernel<<<1, 32, 0, st>>>(d);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof h, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d);
    if (e != cudaSuccess) return npx::set_last_error(NPX_ECUDA, cudaGetErrorString(e));
    *gave_up = h[0];
    *completed = h[1];
    *elapsed_us = h[2];
    return NPX_OK;
}
