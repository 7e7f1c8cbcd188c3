// npx_world.cpp -- host side of libnpx: the C-ABI of include/npx.h.
//
// Construction follows the paper's robot API (NeoPhysIx Sec. IV and Appendix: bodies made of
// mass points, connectBodies, createJoint, finalizeConstruction); npx_scenes_add is the batched
// equivalent for many scenes at once.  finalize packs every scene into the structure-of-arrays
// device layout of npx_internal.h and orders the scenes by point count for the persistent step
// kernel.  Stepping queues chunks of the step kernel on the world's stream, captured once per
// step count into a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/npx.h"
#include "../../include/npx_mlp.h"
#include "npx_internal.h"

namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CUDA_TRY(call)                                                                        \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(NPX_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                        __LINE__);                                                            \
    } while (0)

struct Body {
    std::vector<float> xyz, m;
    int sensor = -1;
};

struct JointDef {
    int b1, b2;
    float anchor[3], axis[3], lo, hi;
};

// A scene built body by body (the paper's API); converted to a Flat scene at finalize.
struct Build {
    std::vector<Body> bodies;
    std::vector<std::pair<int, int>> glue;
    std::vector<JointDef> joints;
};

// A scene in link form: link 0 root, link k hangs from parent[k] < k by joint k-1.
struct Flat {
    std::vector<int> parent, sensor;
    std::vector<float> anchor, axis, lo, hi;
    std::vector<float> p0, m;
    std::vector<int> plink;
};

struct DevBuf {
    void *p = nullptr;
    size_t n = 0;
};

}  // namespace

struct npx_world {
    npx_world_desc desc{};
    cudaStream_t stream = nullptr;
    cudaStream_t own_stream = nullptr;  // created when the caller passes no stream
    int device = 0, n_sm = 0;
    // construction
    std::vector<Build> builds;
    std::vector<Flat> flats;
    std::vector<uint8_t> kind;          // 0 undefined, 1 build, 2 flat
    std::vector<float> mu;
    std::vector<int> hmap;
    std::vector<float> hm_host;         // height maps until finalize uploads them
    bool finalized = false;
    // packed sizes
    int S = 0, P = 0, L = 0, J = 0, max_points = 0, max_links = 0;
    std::vector<int> link_off, point_off;
    // points are stored per scene in ascending construction-frame height; perm maps a stored
    // (global) point index to the caller's index
    std::vector<int> perm;
    // device
    std::vector<DevBuf> bufs;
    npx::WorldDev W{};
    long long *d_step = nullptr;
    float *d_stage = nullptr;           // state staging, AoS blocks [16 * S]
    uint8_t *d_kstage = nullptr;        // contact-flag staging in the caller's order [P]
    int *d_perm = nullptr;              // [P] caller index of each stored point
    float *d_points = nullptr;          // points_read staging [3 * max_points]
    long long step = 0;
    // launch shape
    npx::LaunchCfg cfg{32, 4, 0};       // whole-world launch shape (single steps, the fallback)
    // chunked stepping runs one launch per size class: a slice of the schedule (scenes of similar
    // point counts, most points first) with its own shared-memory slots and launch shape
    struct SizeClass {
        int start, count, max_points, max_links;   // slice of the schedule and its largest scene
        int qi;                                    // its work-queue counter
        npx::LaunchCfg cfg;
    };
    std::vector<SizeClass> classes;
    // classes run concurrently on the world's stream and up to kAuxStreams more (forked and joined
    // with events), so that one class's last wave overlaps the next class's launch
    std::vector<cudaStream_t> aux;
    cudaEvent_t ev_fork = nullptr;
    std::vector<cudaEvent_t> ev_join;
    std::vector<int> order_host;        // the schedule: scenes by point count, descending
    int chunk = 1000;
    bool graphs = true;
    std::map<int, cudaGraphExec_t> graph_cache;
    long long launches = 0;
    int act_mode = NPX_ACT_HOLD;
    bool uniform_links = true;          // every scene has max_links links
    int sensor_bits = 0;                // highest contact-sensor bit + 1
    // surrogate-step buffers, allocated on first use
    struct {
        bool ready = false;
        float *F0 = nullptr, *C0 = nullptr;   // raw features and CoG (x, y) before a collected step
        npx::SurCache cache{};
        float *nx = nullptr;                  // candidate next states [16 * S]
        uint8_t *applied = nullptr;           // [S]
        uint32_t *sens_new = nullptr;         // [S]
        int *list = nullptr, *count = nullptr;
        int *fb = nullptr;                    // [S] windows of each scene that fell back
        int max_changed = 0;                  // fallback when more sensor bits change (32: never)
        // posed-shape cache of every scene (read at the entry of the surrogate's plain launches);
        // current when scache_ok: written by a launch over all scenes since the last change of
        // joint angles from outside the surrogate's own launches
        float4 *scache = nullptr;
        int scache_mp = 0, scache_mt = 0, scache_ml = 0;
        bool scache_ok = false;
        long long *total = nullptr;
        cudaEvent_t ev_w = nullptr, ev_n = nullptr;
        int rows = 0;
        // the shape cache holds the shapes of step cache_at under state generation cache_gen
        long long cache_at = -1;
        unsigned long long cache_gen = ~0ull;
    } sg;
    unsigned long long state_gen = 0;   // counts the caller's state writes
    size_t alist_n = 0;                 // entries allocated for the arenas' pair lists
    CUtensorMap hm_tmap{};              // TMA map of the height maps (W.hm_tmap_h points here)
    // angular velocity and contact sensors are derived from the state: after a state write they
    // are recomputed when first needed (a step recomputes them anyway)
    bool derived_stale = false;
    cudaEvent_t ev_copied = nullptr;    // a state write's host arrays have been read
};

namespace {

template <class T>
int dev_alloc(npx_world *w, T **out, size_t count) {
    void *p = nullptr;
    size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) return fail(NPX_ENOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    w->bufs.push_back({p, bytes});
    *out = static_cast<T *>(p);
    return NPX_OK;
}

int check_world(npx_world *w) {
    if (!w) return fail(NPX_EINVAL, "null world");
    return NPX_OK;
}

int check_building(npx_world *w, int scene) {
    if (int rc = check_world(w)) return rc;
    if (w->finalized) return fail(NPX_ESTATE, "world already finalized");
    if (scene < 0 || scene >= w->desc.n_scenes) return fail(NPX_EINVAL, "scene %d out of range", scene);
    return NPX_OK;
}

int check_ready(npx_world *w) {
    if (int rc = check_world(w)) return rc;
    if (!w->finalized) return fail(NPX_ESTATE, "world not finalized");
    return NPX_OK;
}

Build &build_of(npx_world *w, int scene) {
    if (w->kind[scene] != 1) {
        w->builds[scene] = Build{};
        w->flats[scene] = Flat{};
        w->kind[scene] = 1;
    }
    return w->builds[scene];
}

int find_root(std::vector<int> &par, int x) {
    while (par[x] != x) x = par[x] = par[par[x]];
    return x;
}

// Turn a body-by-body scene into link form: links = groups of glued bodies; the root link holds
// body 0; joints orient the link tree away from it (body1 on the parent side).
int build_to_flat(const Build &b, int scene, Flat &f) {
    const int nb = (int)b.bodies.size();
    if (nb == 0) return fail(NPX_EINVAL, "scene %d has no bodies", scene);
    std::vector<int> uf(nb);
    std::iota(uf.begin(), uf.end(), 0);
    for (auto &g : b.glue) uf[find_root(uf, g.second)] = find_root(uf, g.first);
    std::vector<int> comp(nb, -1), comp_root;
    for (int i = 0; i < nb; ++i) {
        int r = find_root(uf, i);
        if (comp[r] < 0) { comp[r] = (int)comp_root.size(); comp_root.push_back(r); }
        comp[i] = comp[r];
    }
    const int nc = (int)comp_root.size();
    if ((int)b.joints.size() != nc - 1)
        return fail(NPX_EINVAL, "scene %d: %d links need %d joints, got %zu", scene, nc, nc - 1,
                    b.joints.size());
    // breadth-first order from the root link
    std::vector<int> order{comp[0]}, link_of(nc, -1), pj(nc, -1);
    link_of[comp[0]] = 0;
    for (size_t h = 0; h < order.size(); ++h) {
        for (int j = 0; j < (int)b.joints.size(); ++j) {
            const JointDef &jd = b.joints[j];
            int c1 = comp[jd.b1], c2 = comp[jd.b2];
            if (c1 != order[h]) continue;
            if (link_of[c2] >= 0)
                return fail(NPX_EINVAL, "scene %d: joint %d closes a loop", scene, j);
            link_of[c2] = (int)order.size();
            pj[link_of[c2]] = j;
            order.push_back(c2);
        }
    }
    if ((int)order.size() != nc)
        return fail(NPX_EINVAL, "scene %d: joints do not connect every link to the root "
                                "(body1 must be on the root side)", scene);
    f = Flat{};
    f.parent.assign(nc, -1);
    f.sensor.assign(nc, -1);
    f.anchor.assign(3 * nc, 0.f);
    f.axis.assign(3 * nc, 0.f);
    f.lo.assign(nc, 0.f);
    f.hi.assign(nc, 0.f);
    for (int k = 1; k < nc; ++k) {
        const JointDef &jd = b.joints[pj[k]];
        f.parent[k] = link_of[comp[jd.b1]];
        for (int a = 0; a < 3; ++a) { f.anchor[3 * k + a] = jd.anchor[a]; f.axis[3 * k + a] = jd.axis[a]; }
        f.lo[k] = jd.lo;
        f.hi[k] = jd.hi;
    }
    for (int k = 0; k < nc; ++k) {
        for (int i = 0; i < nb; ++i) {
            if (comp[i] != order[k]) continue;
            const Body &bd = b.bodies[i];
            if (bd.sensor >= 0) f.sensor[k] = bd.sensor;
            for (size_t p = 0; p < bd.m.size(); ++p) {
                f.p0.insert(f.p0.end(), bd.xyz.begin() + 3 * p, bd.xyz.begin() + 3 * p + 3);
                f.m.push_back(bd.m[p]);
                f.plink.push_back(k);
            }
        }
    }
    return NPX_OK;
}

int check_flat(const Flat &f, int scene) {
    const int nl = (int)f.parent.size(), np = (int)f.m.size();
    if (nl < 1 || nl > NPX_MAX_LINKS) return fail(NPX_ERANGE, "scene %d: %d links (1..%d)", scene, nl, NPX_MAX_LINKS);
    if (np < 1 || np > NPX_MAX_POINTS) return fail(NPX_ERANGE, "scene %d: %d points (1..%d)", scene, np, NPX_MAX_POINTS);
    if (f.parent[0] != -1) return fail(NPX_EINVAL, "scene %d: link 0 must be the root", scene);
    for (int k = 1; k < nl; ++k) {
        if (f.parent[k] < 0 || f.parent[k] >= k) return fail(NPX_EINVAL, "scene %d: link %d parent %d not in [0,%d)", scene, k, f.parent[k], k);
        double n2 = 0;
        for (int a = 0; a < 3; ++a) n2 += (double)f.axis[3 * k + a] * f.axis[3 * k + a];
        if (!(n2 > 0.0) || !std::isfinite(n2)) return fail(NPX_EINVAL, "scene %d: link %d has a zero axis", scene, k);
        if (!(f.lo[k] <= f.hi[k])) return fail(NPX_EINVAL, "scene %d: link %d limits lo > hi", scene, k);
    }
    for (int k = 0; k < nl; ++k)
        if (f.sensor[k] >= NPX_MAX_SENSORS) return fail(NPX_ERANGE, "scene %d: sensor bit %d >= %d", scene, f.sensor[k], NPX_MAX_SENSORS);
    for (int i = 0; i < np; ++i) {
        if (!(f.m[i] > 0.f) || !std::isfinite(f.m[i])) return fail(NPX_EINVAL, "scene %d: point %d mass must be > 0", scene, i);
        if (f.plink[i] < 0 || f.plink[i] >= nl) return fail(NPX_EINVAL, "scene %d: point %d link out of range", scene, i);
        for (int a = 0; a < 3; ++a)
            if (!std::isfinite(f.p0[3 * i + a])) return fail(NPX_EINVAL, "scene %d: point %d not finite", scene, i);
    }
    return NPX_OK;
}

// launch shape for the scenes of W's schedule (count of them): checks the lanes per scene against
// the largest scene, and sizes the grid to what is resident and what is needed
npx::LaunchCfg clamp_cfg_for(npx_world *w, const npx::WorldDev &W, int count, npx::LaunchCfg c, int *rc) {
    *rc = NPX_OK;
    if (W.arena > 1 && c.lps * W.arena > 32) {
        *rc = fail(NPX_ERANGE, "an arena of %d robots is one warp: at most %d lanes per scene", W.arena, 32 / W.arena);
        return c;
    }
    if (W.max_points > 64 * c.lps) {
        *rc = fail(NPX_ERANGE, "%d points per scene exceed 64 per lane at %d lanes per scene",
                   W.max_points, c.lps);
        return c;
    }
    cudaError_t e;
    int nb = npx::step_blocks_per_sm(W, c.lps, c.wpb, &e);
    if (e != cudaSuccess) { *rc = fail(NPX_ECUDA, "occupancy query: %s", cudaGetErrorString(e)); return c; }
    if (nb < 1) { *rc = fail(NPX_ERANGE, "launch shape lps=%d wpb=%d does not fit on an SM", c.lps, c.wpb); return c; }
    const int per_block = c.wpb * (32 / c.lps);
    const int need = (count + per_block - 1) / per_block;
    const int full = nb * w->n_sm;
    if (c.blocks <= 0 || c.blocks > full) c.blocks = full;
    c.blocks = std::max(1, std::min(c.blocks, need));
    return c;
}

npx::LaunchCfg clamp_cfg(npx_world *w, npx::LaunchCfg c, int *rc) { return clamp_cfg_for(w, w->W, w->S, c, rc); }

// the world as one class's launch sees it: its slice of the schedule, its slot sizes and its own
// work-queue counter (built from the current world, so that later changes -- actuators, state --
// reach every class)
npx::WorldDev class_world(const npx_world *w, const npx_world::SizeClass &c) {
    npx::WorldDev W = w->W;
    W.order = w->W.order + c.start;
    W.n_sched = c.count;
    W.sched_count = nullptr;
    W.max_points = c.max_points;
    W.max_links = c.max_links;
    W.queue = w->W.queue + c.qi;
    return W;
}

// default shape for scenes of up to max_points points: the narrowest group that holds them,
// at least 16 lanes, 4 warps per block
npx::LaunchCfg default_shape(int max_points) {
    int lps = 8;
    while (lps < 32 && max_points > 64 * lps) lps *= 2;
    return {std::max(lps, 16), 4, 0};
}

// Size classes of the schedule (scenes by point count, descending): runs whose smallest scene has
// at least 1/kClassRatio the points of the largest, so that a class's shared-memory slots (sized
// for its largest scene) waste little; a class of fewer than min_count scenes joins the class
// before it (or, the first, the one after).  A world of equal scenes has one class, the whole
// world.
// (ratio 1.3 and min_count S / 64 measured best on the uneven 65,536-scene mix against 1.15 / S /
// 256, 1.5 / S / 32 and 2 / S / 64)
constexpr double kClassRatio = 1.3;
constexpr int kMaxClasses = 64;   // work-queue counters
constexpr int kAuxStreams = 3;

int build_classes(npx_world *w, bool split) {
    w->classes.clear();
    if (w->W.arena > 1) split = false;   // an arena's robots run in one warp of one launch
    const int S = w->S;
    const std::vector<int> &order = w->order_host;
    auto pts = [&](int s) { return w->point_off[s + 1] - w->point_off[s]; };
    auto lnk = [&](int s) { return w->link_off[s + 1] - w->link_off[s]; };
    std::vector<std::pair<int, int>> ranges;
    if (split) {
        const int min_count = std::max(256, S / 64);
        for (int start = 0; start < S;) {
            const int top = pts(order[start]);
            int end = start + 1;
            while (end < S && (double)pts(order[end]) * kClassRatio >= (double)top) ++end;
            if (!ranges.empty() && end - start < min_count) ranges.back().second = end;
            else ranges.push_back({start, end});
            start = end;
        }
        if (ranges.size() > 1 && ranges[0].second - ranges[0].first < min_count) {
            ranges[1].first = ranges[0].first;
            ranges.erase(ranges.begin());
        }
        // at most kMaxClasses: join the smallest class with its smaller-scene neighbour
        while ((int)ranges.size() > kMaxClasses) {
            size_t k = 0;
            for (size_t i = 1; i + 1 < ranges.size(); ++i)
                if (ranges[i].second - ranges[i].first < ranges[k].second - ranges[k].first) k = i;
            if (k + 1 == ranges.size()) --k;
            ranges[k].second = ranges[k + 1].second;
            ranges.erase(ranges.begin() + (long)k + 1);
        }
    } else {
        ranges.push_back({0, S});
    }
    // side streams and events for concurrent class launches
    if (ranges.size() > 1 && w->aux.empty()) {
        CUDA_TRY(cudaEventCreateWithFlags(&w->ev_fork, cudaEventDisableTiming));
        for (int a = 0; a < kAuxStreams; ++a) {
            cudaStream_t st;
            cudaEvent_t ev;
            CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
            w->aux.push_back(st);
            CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
            w->ev_join.push_back(ev);
        }
    }
    for (const auto &r : ranges) {
        npx_world::SizeClass c;
        c.qi = (int)w->classes.size();
        c.start = r.first;
        c.count = r.second - r.first;
        c.max_points = 1;
        c.max_links = 1;
        for (int i = r.first; i < r.second; ++i) {
            c.max_points = std::max(c.max_points, pts(order[i]));
            c.max_links = std::max(c.max_links, lnk(order[i]));
        }
        if (ranges.size() == 1) {
            c.cfg = w->cfg;
        } else {
            int rc;
            c.cfg = clamp_cfg_for(w, class_world(w, c), c.count, default_shape(c.max_points), &rc);
            if (rc) return rc;
        }
        w->classes.push_back(c);
    }
    return NPX_OK;
}

void clear_graphs(npx_world *w) {
    for (auto &kv : w->graph_cache) cudaGraphExecDestroy(kv.second);
    w->graph_cache.clear();
}

// angular velocity and contact sensors consistent with the state (after a state write)
int ensure_derived(npx_world *w) {
    if (!w->derived_stale) return NPX_OK;
    CUDA_TRY(npx::launch_refresh(w->W, w->stream));
    w->derived_stale = false;
    return NPX_OK;
}

int enqueue_steps(npx_world *w, int n) {
    const int nk = (int)w->classes.size();
    const int na = std::min(nk - 1, (int)w->aux.size());   // side streams in use
    for (int done = 0; done < n;) {
        const int nc = std::min(w->chunk, n - done);
        // every class reads the same step counter; it advances after all of them.  Classes go
        // round-robin to the world's stream and the side streams, which fork from it and join it.
        if (na > 0) {
            CUDA_TRY(cudaEventRecord(w->ev_fork, w->stream));
            for (int a = 0; a < na; ++a) CUDA_TRY(cudaStreamWaitEvent(w->aux[a], w->ev_fork, 0));
        }
        for (int i = 0; i < nk; ++i) {
            const auto &c = w->classes[i];
            const int k = na > 0 ? i % (na + 1) : 0;
            CUDA_TRY(npx::launch_step(class_world(w, c), c.cfg, nc, k == 0 ? w->stream : w->aux[k - 1]));
        }
        for (int a = 0; a < na; ++a) {
            CUDA_TRY(cudaEventRecord(w->ev_join[a], w->aux[a]));
            CUDA_TRY(cudaStreamWaitEvent(w->stream, w->ev_join[a], 0));
        }
        CUDA_TRY(npx::launch_advance(w->d_step, nc, w->stream));
        done += nc;
    }
    return NPX_OK;
}

struct BlobLayout {
    size_t st, theta, omega, kappa, sensors, status, gp_pc, gp_acc, gp_k, end;
};

BlobLayout blob_layout(const npx_world *w) {
    BlobLayout b;
    b.st = 64;
    b.theta = b.st + sizeof(float) * (size_t)npx::ST_N * w->S;
    b.omega = b.theta + sizeof(float) * (size_t)w->J;
    b.sensors = b.omega + sizeof(float) * 3 * (size_t)w->S;
    b.status = b.sensors + sizeof(uint32_t) * (size_t)w->S;
    b.kappa = b.status + sizeof(uint32_t) * (size_t)w->S;
    b.gp_pc = b.kappa + (size_t)w->P;        // the machine-code controller's state
    b.gp_acc = b.gp_pc + (size_t)w->S;
    b.gp_k = b.gp_acc + (size_t)w->S;
    b.end = b.gp_k + (size_t)w->J;
    return b;
}

const uint64_t kBlobMagic = 0x315850584e504e47ull;

}  // namespace

namespace {

int surrogate_dims(npx_world *w, int *nf, int *nt) {
    if (!w->uniform_links) return fail(NPX_EINVAL, "surrogate features need scenes with equal link counts");
    const int NL = w->max_links;
    *nf = 14 * NL - 1 + w->sensor_bits;
    *nt = 13 * NL;
    return NPX_OK;
}

int surrogate_buffers(npx_world *w) {
    if (w->sg.ready) return NPX_OK;
    int nf, nt;
    if (int rc = surrogate_dims(w, &nf, &nt)) return rc;
    const int rows = (w->S + 127) / 128 * 128;
    npx::SurCache &C = w->sg.cache;
    int rc, *d_max = nullptr;
    if ((rc = dev_alloc(w, &w->sg.F0, (size_t)w->S * nf)) || (rc = dev_alloc(w, &w->sg.C0, 2 * (size_t)w->S)) ||
        (rc = dev_alloc(w, &w->sg.list, w->S)) || (rc = dev_alloc(w, &w->sg.count, 1)) ||
        (rc = dev_alloc(w, &w->sg.total, 1)) || (rc = dev_alloc(w, &C.lk, 2 * (size_t)w->S * w->max_links)) ||
        (rc = dev_alloc(w, &C.inert, 12 * (size_t)w->S)) || (rc = dev_alloc(w, &C.nsp_s, w->S)) ||
        (rc = dev_alloc(w, &d_max, 1)) || (rc = dev_alloc(w, &w->sg.nx, 16 * (size_t)w->S)) ||
        (rc = dev_alloc(w, &w->sg.applied, w->S)) || (rc = dev_alloc(w, &w->sg.sens_new, w->S)) ||
        (rc = dev_alloc(w, &w->sg.fb, w->S)))
        return rc;
    w->sg.scache_mp = w->max_points;
    w->sg.scache_mt = (w->max_points + 3) / 4;   // tiles at the fewest lanes per scene (4)
    w->sg.scache_ml = w->max_links;
    if ((rc = dev_alloc(w, &w->sg.scache,
                        (size_t)w->S * (w->sg.scache_mp + 2 * w->sg.scache_mt + 5 + 2 * w->sg.scache_ml))))
        return rc;
    w->sg.scache_ok = false;
    CUDA_TRY(cudaMemsetAsync(w->sg.count, 0, sizeof(int), w->stream));
    CUDA_TRY(cudaMemsetAsync(w->sg.fb, 0, sizeof(int) * (size_t)w->S, w->stream));
    CUDA_TRY(cudaMemsetAsync(d_max, 0, sizeof(int), w->stream));
    CUDA_TRY(npx::launch_sensor_points(w->W, C.nsp_s, d_max, w->stream));
    int nsp = 0;
    CUDA_TRY(cudaMemcpyAsync(&nsp, d_max, sizeof(int), cudaMemcpyDeviceToHost, w->stream));
    CUDA_TRY(cudaStreamSynchronize(w->stream));
    if ((rc = dev_alloc(w, &C.spt, (size_t)w->S * std::max(nsp, 1))) ||
        (rc = dev_alloc(w, &C.sidx, (size_t)w->S * std::max(nsp, 1))))
        return rc;
    C.nsp = std::max(nsp, 1);
    CUDA_TRY(npx::launch_sensor_index(w->W, C, w->stream));
    C.nl = w->max_links;
    CUDA_TRY(cudaEventCreateWithFlags(&w->sg.ev_w, cudaEventDisableTiming));
    CUDA_TRY(cudaEventCreateWithFlags(&w->sg.ev_n, cudaEventDisableTiming));
    w->sg.rows = rows;
    w->sg.ready = true;
    return NPX_OK;
}

}  // namespace

int npx::set_last_error(int code, const char *msg) {
    g_err = msg;
    return code;
}

extern "C" {

const char *npx_last_error(void) { return g_err.c_str(); }

int npx_world_create(const npx_world_desc *d, npx_world **out) {
    if (!d || !out) return fail(NPX_EINVAL, "null argument");
    *out = nullptr;
    if (d->n_scenes < 1) return fail(NPX_EINVAL, "n_scenes must be >= 1");
    if (!(d->dt > 0.f) || !std::isfinite(d->dt)) return fail(NPX_EINVAL, "dt must be > 0");
    if (d->joint_update_steps < 1) return fail(NPX_EINVAL, "joint_update_steps must be >= 1");
    if (!(d->contact_omega > 0.f) || !(d->contact_zeta >= 0.f))
        return fail(NPX_EINVAL, "contact_omega must be > 0 and contact_zeta >= 0");
    if (d->hm_count < 0) return fail(NPX_EINVAL, "hm_count < 0");
    if (d->hm_count > 0 && (!d->hm_data || d->hm_nx < 1 || d->hm_ny < 1 || !(d->hm_scale > 0.f)))
        return fail(NPX_EINVAL, "height maps need data, nx, ny >= 1 and scale > 0");
    if (d->device < 0) return fail(NPX_EINVAL, "device %d out of range", d->device);
    npx_world *w = new (std::nothrow) npx_world();
    if (!w) return fail(NPX_ENOMEM, "out of host memory");
    w->desc = *d;
    w->desc.hm_data = nullptr;
    w->device = d->device;
    w->stream = static_cast<cudaStream_t>(d->stream);
    const int S = d->n_scenes;
    w->builds.resize(S);
    w->flats.resize(S);
    w->kind.assign(S, 0);
    w->mu.assign(S, 0.5f);
    w->hmap.assign(S, d->hm_count > 0 ? 0 : -1);
    // the caller's height maps are copied now and uploaded at finalize
    if (d->hm_count > 0)
        w->hm_host.assign(d->hm_data, d->hm_data + (size_t)d->hm_count * d->hm_ny * d->hm_nx);
    *out = w;
    return NPX_OK;
}

int npx_world_destroy(npx_world *w) {
    if (!w) return NPX_OK;
    if (!w->bufs.empty()) {
        cudaSetDevice(w->device);
        if (w->finalized) cudaStreamSynchronize(w->stream);
        clear_graphs(w);
        for (auto &b : w->bufs) cudaFree(b.p);
    }
    if (w->sg.ev_w) cudaEventDestroy(w->sg.ev_w);
    if (w->sg.ev_n) cudaEventDestroy(w->sg.ev_n);
    for (cudaStream_t st : w->aux) cudaStreamDestroy(st);
    if (w->ev_copied) cudaEventDestroy(w->ev_copied);
    for (cudaEvent_t ev : w->ev_join) cudaEventDestroy(ev);
    if (w->ev_fork) cudaEventDestroy(w->ev_fork);
    if (w->own_stream) cudaStreamDestroy(w->own_stream);
    delete w;
    return NPX_OK;
}

int npx_body_add_pointcloud(npx_world *w, int scene, const float *xyz, const float *mass,
                            float total_mass, int n, int *out_body) {
    if (int rc = check_building(w, scene)) return rc;
    if (!xyz || n < 1) return fail(NPX_EINVAL, "need n >= 1 points");
    if (!mass && !(total_mass > 0.f)) return fail(NPX_EINVAL, "total_mass must be > 0");
    Build &b = build_of(w, scene);
    Body bd;
    bd.xyz.assign(xyz, xyz + 3 * (size_t)n);
    if (mass) bd.m.assign(mass, mass + n);
    else bd.m.assign(n, total_mass / (float)n);
    b.bodies.push_back(std::move(bd));
    if (out_body) *out_body = (int)b.bodies.size() - 1;
    return NPX_OK;
}

int npx_body_connect(npx_world *w, int scene, int body1, int body2) {
    if (int rc = check_building(w, scene)) return rc;
    if (w->kind[scene] != 1) return fail(NPX_ESTATE, "scene %d has no bodies", scene);
    Build &b = w->builds[scene];
    const int nb = (int)b.bodies.size();
    if (body1 < 0 || body1 >= nb || body2 < 0 || body2 >= nb) return fail(NPX_EINVAL, "body id out of range");
    b.glue.push_back({body1, body2});
    return NPX_OK;
}

int npx_joint_add(npx_world *w, int scene, int body1, int body2, const float anchor[3],
                  const float axis[3], float lo, float hi, int *out_joint) {
    if (int rc = check_building(w, scene)) return rc;
    if (w->kind[scene] != 1) return fail(NPX_ESTATE, "scene %d has no bodies", scene);
    if (!anchor || !axis) return fail(NPX_EINVAL, "null anchor or axis");
    Build &b = w->builds[scene];
    const int nb = (int)b.bodies.size();
    if (body1 < 0 || body1 >= nb || body2 < 0 || body2 >= nb || body1 == body2)
        return fail(NPX_EINVAL, "body id out of range");
    if (!(lo <= hi)) return fail(NPX_EINVAL, "joint limits lo > hi");
    JointDef j{body1, body2, {anchor[0], anchor[1], anchor[2]}, {axis[0], axis[1], axis[2]}, lo, hi};
    b.joints.push_back(j);
    if (out_joint) *out_joint = (int)b.joints.size() - 1;
    return NPX_OK;
}

int npx_sensor_add(npx_world *w, int scene, int body, int bit) {
    if (int rc = check_building(w, scene)) return rc;
    if (w->kind[scene] != 1) return fail(NPX_ESTATE, "scene %d has no bodies", scene);
    Build &b = w->builds[scene];
    if (body < 0 || body >= (int)b.bodies.size()) return fail(NPX_EINVAL, "body id out of range");
    if (bit < 0 || bit >= NPX_MAX_SENSORS) return fail(NPX_ERANGE, "sensor bit %d out of range", bit);
    b.bodies[body].sensor = bit;
    return NPX_OK;
}

int npx_scene_set_friction(npx_world *w, int scene, float mu) {
    if (int rc = check_building(w, scene)) return rc;
    if (!(mu >= 0.f) || !std::isfinite(mu)) return fail(NPX_EINVAL, "mu must be >= 0");
    w->mu[scene] = mu;
    return NPX_OK;
}

int npx_scene_set_heightmap(npx_world *w, int scene, int hm) {
    if (int rc = check_building(w, scene)) return rc;
    if (hm < -1 || hm >= w->desc.hm_count) return fail(NPX_EINVAL, "height map %d out of range", hm);
    w->hmap[scene] = hm;
    return NPX_OK;
}

int npx_scene_clone(npx_world *w, int src, int first_dst, int count) {
    if (int rc = check_building(w, src)) return rc;
    if (count < 0 || first_dst < 0 || (long long)first_dst + count > w->desc.n_scenes)
        return fail(NPX_EINVAL, "clone range out of bounds");
    if (w->kind[src] == 0) return fail(NPX_ESTATE, "scene %d is not defined", src);
    for (int d = first_dst; d < first_dst + count; ++d) {
        if (d == src) continue;
        w->kind[d] = w->kind[src];
        if (w->kind[src] == 1) w->builds[d] = w->builds[src];
        else w->flats[d] = w->flats[src];
        w->mu[d] = w->mu[src];
        w->hmap[d] = w->hmap[src];
    }
    return NPX_OK;
}

int npx_scenes_add(npx_world *w, const npx_scene_batch *b) {
    if (int rc = check_world(w)) return rc;
    if (w->finalized) return fail(NPX_ESTATE, "world already finalized");
    if (!b || !b->link_off || !b->point_off || !b->parent || !b->anchor || !b->axis || !b->lo ||
        !b->hi || !b->sensor || !b->p0 || !b->m || !b->plink || !b->mu)
        return fail(NPX_EINVAL, "null array in scene batch");
    if (b->count < 0 || b->first < 0 || (long long)b->first + b->count > w->desc.n_scenes)
        return fail(NPX_EINVAL, "scene range [%d, %d) out of bounds", b->first, b->first + b->count);
    if (b->link_off[0] != 0 || b->point_off[0] != 0) return fail(NPX_EINVAL, "offsets must start at 0");
    for (int s = 0; s < b->count; ++s) {
        const int l0 = b->link_off[s], l1 = b->link_off[s + 1];
        const int p0 = b->point_off[s], p1 = b->point_off[s + 1];
        if (l1 <= l0 || p1 <= p0) return fail(NPX_EINVAL, "scene %d: empty links or points", b->first + s);
        const int sc = b->first + s;
        Flat f;
        f.parent.assign(b->parent + l0, b->parent + l1);
        f.sensor.assign(b->sensor + l0, b->sensor + l1);
        f.anchor.assign(b->anchor + 3 * (size_t)l0, b->anchor + 3 * (size_t)l1);
        f.axis.assign(b->axis + 3 * (size_t)l0, b->axis + 3 * (size_t)l1);
        f.lo.assign(b->lo + l0, b->lo + l1);
        f.hi.assign(b->hi + l0, b->hi + l1);
        f.p0.assign(b->p0 + 3 * (size_t)p0, b->p0 + 3 * (size_t)p1);
        f.m.assign(b->m + p0, b->m + p1);
        f.plink.assign(b->plink + p0, b->plink + p1);
        if (int rc = check_flat(f, sc)) return rc;
        w->flats[sc] = std::move(f);
        w->builds[sc] = Build{};
        w->kind[sc] = 2;
        if (!(b->mu[s] >= 0.f) || !std::isfinite(b->mu[s])) return fail(NPX_EINVAL, "scene %d: mu must be >= 0", sc);
        w->mu[sc] = b->mu[s];
        const int hm = b->hmap ? b->hmap[s] : (w->desc.hm_count > 0 ? 0 : -1);
        if (hm < -1 || hm >= w->desc.hm_count) return fail(NPX_EINVAL, "scene %d: height map %d out of range", sc, hm);
        w->hmap[sc] = hm;
    }
    return NPX_OK;
}

int npx_world_finalize(npx_world *w) {
    if (int rc = check_world(w)) return rc;
    if (w->finalized) return fail(NPX_ESTATE, "world already finalized");
    const int S = w->desc.n_scenes;
    for (int s = 0; s < S; ++s) {
        if (w->kind[s] == 0) return fail(NPX_ESTATE, "scene %d is not defined", s);
        if (w->kind[s] == 1) {
            if (int rc = build_to_flat(w->builds[s], s, w->flats[s])) return rc;
            if (int rc = check_flat(w->flats[s], s)) return rc;
            w->builds[s] = Build{};
            w->kind[s] = 2;
        }
    }
    // ---- pack
    w->S = S;
    w->link_off.assign(S + 1, 0);
    w->point_off.assign(S + 1, 0);
    for (int s = 0; s < S; ++s) {
        w->link_off[s + 1] = w->link_off[s] + (int)w->flats[s].parent.size();
        w->point_off[s + 1] = w->point_off[s] + (int)w->flats[s].m.size();
        w->max_links = std::max(w->max_links, (int)w->flats[s].parent.size());
        w->max_points = std::max(w->max_points, (int)w->flats[s].m.size());
    }
    w->L = w->link_off[S];
    w->P = w->point_off[S];
    if (w->max_points > 64 * 32)
        return fail(NPX_ERANGE, "a scene has %d points; at most 2048 (64 per lane at 32 lanes per scene)",
                    w->max_points);
    for (int s = 0; s < S; ++s) {
        if (w->link_off[s + 1] - w->link_off[s] != w->max_links) w->uniform_links = false;
        for (int sid : w->flats[s].sensor) w->sensor_bits = std::max(w->sensor_bits, sid + 1);
    }
    w->J = w->L - S;
    std::vector<npx::LinkDev> links(w->L);
    w->perm.assign(w->P, 0);
    // rest-pose CoG of each scene: the kernels sum mass moments about it (a numerical reference
    // only; the results do not depend on it beyond rounding); CoG of each link's points
    std::vector<float> gref(3 * (size_t)S), lcog(3 * (size_t)w->L, 0.f);
    std::vector<float4> p0m(w->P);
    std::vector<uint8_t> plink(w->P);
    for (int s = 0; s < S; ++s) {
        const Flat &f = w->flats[s];
        const int l0 = w->link_off[s], p0 = w->point_off[s], nl = (int)f.parent.size();
        std::vector<int> depth(nl, 0);
        for (int k = 0; k < nl; ++k) {
            npx::LinkDev &ld = links[l0 + k];
            if (k > 0) depth[k] = depth[f.parent[k]] + 1;
            double ux = f.axis[3 * k], uy = f.axis[3 * k + 1], uz = f.axis[3 * k + 2];
            double un = std::sqrt(ux * ux + uy * uy + uz * uz);
            if (k == 0) { ux = 0; uy = 0; uz = 1; un = 1; }
            ld = {f.anchor[3 * k], f.anchor[3 * k + 1], f.anchor[3 * k + 2], f.lo[k],
                  (float)(ux / un), (float)(uy / un), (float)(uz / un), f.hi[k],
                  f.parent[k], f.sensor[k], depth[k], 0};
        }
        {
            double m = 0, g[3] = {0, 0, 0};
            for (size_t i = 0; i < f.m.size(); ++i) {
                m += f.m[i];
                for (int k = 0; k < 3; ++k) g[k] += (double)f.m[i] * f.p0[3 * i + k];
            }
            for (int k = 0; k < 3; ++k) gref[3 * s + k] = (float)(g[k] / m);
            std::vector<double> lm(nl, 0.0), lg(3 * (size_t)nl, 0.0);
            for (size_t i = 0; i < f.m.size(); ++i) {
                lm[f.plink[i]] += f.m[i];
                for (int k = 0; k < 3; ++k) lg[3 * f.plink[i] + k] += (double)f.m[i] * f.p0[3 * i + k];
            }
            for (int k = 0; k < nl; ++k)
                for (int a = 0; a < 3; ++a)
                    lcog[3 * (size_t)(l0 + k) + a] = lm[k] > 0 ? (float)(lg[3 * k + a] / lm[k]) : 0.f;
        }
        // lowest points first: the step kernel stops scanning once the rest is above ground
        std::vector<int> ord(f.m.size());
        std::iota(ord.begin(), ord.end(), 0);
        std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return f.p0[3 * a + 2] < f.p0[3 * b + 2]; });
        for (size_t i = 0; i < f.m.size(); ++i) {
            const int u = ord[i];
            p0m[p0 + i] = make_float4(f.p0[3 * u], f.p0[3 * u + 1], f.p0[3 * u + 2], f.m[u]);
            plink[p0 + i] = (uint8_t)f.plink[u];
            w->perm[p0 + i] = p0 + u;
        }
    }
    // persistent schedule: most points first (longest jobs start first)
    std::vector<int> order(S);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return w->point_off[a + 1] - w->point_off[a] > w->point_off[b + 1] - w->point_off[b];
    });
    // ---- device
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev < 1) return fail(NPX_ECUDA, "no CUDA device: %s", cudaGetErrorString(e));
    if (w->device >= ndev) return fail(NPX_EINVAL, "device %d out of range (%d devices)", w->device, ndev);
    CUDA_TRY(cudaSetDevice(w->device));
    CUDA_TRY(cudaDeviceGetAttribute(&w->n_sm, cudaDevAttrMultiProcessorCount, w->device));
    if (!w->stream) {   // the legacy default stream cannot be captured into graphs
        CUDA_TRY(cudaStreamCreateWithFlags(&w->own_stream, cudaStreamNonBlocking));
        w->stream = w->own_stream;
    }
    npx::WorldDev &W = w->W;
    if (!w->hm_host.empty()) {
        float *hm = nullptr, *hmx = nullptr;
        if (int rc = dev_alloc(w, &hm, w->hm_host.size())) return rc;
        CUDA_TRY(cudaMemcpy(hm, w->hm_host.data(), w->hm_host.size() * sizeof(float), cudaMemcpyHostToDevice));
        const size_t cells = (size_t)w->desc.hm_nx * w->desc.hm_ny;
        std::vector<float> mx(w->desc.hm_count);
        for (int h = 0; h < w->desc.hm_count; ++h)
            mx[h] = *std::max_element(w->hm_host.begin() + h * cells, w->hm_host.begin() + (h + 1) * cells);
        if (int rc = dev_alloc(w, &hmx, mx.size())) return rc;
        CUDA_TRY(cudaMemcpy(hmx, mx.data(), mx.size() * sizeof(float), cudaMemcpyHostToDevice));
        W.hm = hm;
        W.hm_max = hmx;
        W.hm_nx = w->desc.hm_nx;
        W.hm_ny = w->desc.hm_ny;
        npx::encode_hm_tmap(W, w->desc.hm_count, &w->hm_tmap);
        // the dilated map of the cull's local ground bound: radius R cells covers the largest
        // rest-pose radius about the rest CoG, a quarter more for the joints' reach and 4 cells of
        // drift between culls (a larger posed robot falls back to the map's highest cell)
        float r_rest = 0.f;
        for (int s = 0; s < S; ++s)
            for (int i = w->point_off[s]; i < w->point_off[s + 1]; ++i) {
                const float dx = p0m[i].x - gref[3 * s], dy = p0m[i].y - gref[3 * s + 1],
                            dz = p0m[i].z - gref[3 * s + 2];
                r_rest = std::max(r_rest, std::sqrt(dx * dx + dy * dy + dz * dz));
            }
        const int R = std::min((int)std::ceil(1.25f * r_rest * w->desc.hm_scale) + 4,
                               std::max(w->desc.hm_nx, w->desc.hm_ny));
        float *dmax = nullptr, *tmp = nullptr;
        if (int rc = dev_alloc(w, &dmax, w->hm_host.size())) return rc;
        CUDA_TRY(cudaMalloc(&tmp, w->hm_host.size() * sizeof(float)));
        cudaError_t de = npx::launch_hm_dilate(hm, tmp, dmax, w->desc.hm_count, w->desc.hm_ny, w->desc.hm_nx, R,
                                               w->stream);
        if (de == cudaSuccess) de = cudaStreamSynchronize(w->stream);
        cudaFree(tmp);
        if (de != cudaSuccess) return fail(NPX_ECUDA, "height-map dilation: %s", cudaGetErrorString(de));
        W.hm_dmax = dmax;
        W.hm_dr = R;
        w->hm_host.clear();
        w->hm_host.shrink_to_fit();
    }
    W.S = S; W.P = w->P; W.L = w->L; W.J = w->J;
    int *d_lo, *d_po, *d_hmap, *d_order;
    float *d_gref, *d_lcog;
    float4 *d_p0m, *d_act;
    uint8_t *d_plink, *d_kappa;
    npx::LinkDev *d_links;
    float *d_mu, *d_st, *d_theta, *d_omega;
    uint32_t *d_nu, *d_sens, *d_status;
    unsigned int *d_queue;
    uint8_t *d_gp_prog, *d_gp_pc, *d_gp_acc;
    int8_t *d_gp_k;
    int rc = 0;
    if ((rc = dev_alloc(w, &d_lo, S + 1)) || (rc = dev_alloc(w, &d_po, S + 1)) ||
        (rc = dev_alloc(w, &d_hmap, S)) || (rc = dev_alloc(w, &d_order, S)) ||
        (rc = dev_alloc(w, &d_p0m, w->P)) || (rc = dev_alloc(w, &d_plink, w->P)) ||
        (rc = dev_alloc(w, &d_links, w->L)) || (rc = dev_alloc(w, &d_mu, S)) ||
        (rc = dev_alloc(w, &d_act, w->J)) || (rc = dev_alloc(w, &d_nu, w->J)) ||
        (rc = dev_alloc(w, &d_st, (size_t)npx::ST_N * S)) || (rc = dev_alloc(w, &d_theta, w->J)) ||
        (rc = dev_alloc(w, &d_kappa, w->P)) || (rc = dev_alloc(w, &d_gref, 3 * (size_t)S)) ||
        (rc = dev_alloc(w, &d_lcog, 3 * (size_t)w->L)) ||
        (rc = dev_alloc(w, &d_omega, 3 * (size_t)S)) || (rc = dev_alloc(w, &d_sens, S)) ||
        (rc = dev_alloc(w, &d_status, S)) || (rc = dev_alloc(w, &d_queue, kMaxClasses)) ||
        (rc = dev_alloc(w, &w->d_step, 1)) || (rc = dev_alloc(w, &w->d_stage, 16 * (size_t)S)) ||
        (rc = dev_alloc(w, &w->d_kstage, w->P)) || (rc = dev_alloc(w, &w->d_perm, w->P)) ||
        (rc = dev_alloc(w, &w->d_points, 3 * (size_t)w->max_points)) ||
        (rc = dev_alloc(w, &d_gp_prog, 32 * (size_t)S)) || (rc = dev_alloc(w, &d_gp_pc, S)) ||
        (rc = dev_alloc(w, &d_gp_acc, S)) || (rc = dev_alloc(w, &d_gp_k, w->J)))
        return rc;
    CUDA_TRY(cudaMemset(d_gp_prog, 0, 32 * (size_t)S));
    CUDA_TRY(cudaMemset(d_gp_pc, 0, S));
    CUDA_TRY(cudaMemset(d_gp_acc, 0, S));
    CUDA_TRY(cudaMemset(d_gp_k, 0, std::max(w->J, 1)));
    CUDA_TRY(cudaMemcpy(d_lo, w->link_off.data(), sizeof(int) * (S + 1), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(d_po, w->point_off.data(), sizeof(int) * (S + 1), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(d_hmap, w->hmap.data(), sizeof(int) * S, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(d_order, order.data(), sizeof(int) * S, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(d_p0m, p0m.data(), sizeof(float4) * w->P, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(d_plink, plink.data(), w->P, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(d_links, links.data(), sizeof(npx::LinkDev) * w->L, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(d_mu, w->mu.data(), sizeof(float) * S, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(d_gref, gref.data(), sizeof(float) * 3 * S, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(d_lcog, lcog.data(), sizeof(float) * 3 * w->L, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(w->d_perm, w->perm.data(), sizeof(int) * w->P, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemset(d_act, 0, sizeof(float4) * std::max(w->J, 1)));
    CUDA_TRY(cudaMemset(d_nu, 0, sizeof(uint32_t) * std::max(w->J, 1)));
    CUDA_TRY(cudaMemset(d_theta, 0, sizeof(float) * std::max(w->J, 1)));
    CUDA_TRY(cudaMemset(w->d_step, 0, sizeof(long long)));
    W.link_off = d_lo; W.point_off = d_po; W.p0m = d_p0m; W.plink = d_plink; W.links = d_links;
    W.gref = d_gref;
    W.link_cog = d_lcog;
    W.mu = d_mu; W.hmap = d_hmap;
    W.hm_nx = w->desc.hm_nx; W.hm_ny = w->desc.hm_ny;
    W.hm_scale = w->desc.hm_scale; W.hm_ox = w->desc.hm_origin[0]; W.hm_oy = w->desc.hm_origin[1];
    W.dt = w->desc.dt;
    W.gx = w->desc.gravity[0]; W.gy = w->desc.gravity[1]; W.gz = w->desc.gravity[2];
    W.K = w->desc.joint_update_steps;
    W.kw2 = w->desc.contact_omega * w->desc.contact_omega;
    W.kc = 2.f * w->desc.contact_zeta * w->desc.contact_omega;
    W.act_mode = NPX_ACT_HOLD;
    W.act = d_act; W.act_nu = d_nu;
    W.st = d_st; W.theta = d_theta; W.kappa = d_kappa; W.omega = d_omega;
    W.sensors = d_sens; W.status = d_status;
    W.order = d_order; W.n_sched = S; W.sched_count = nullptr;
    W.max_points = w->max_points; W.max_links = w->max_links;
    W.step = w->d_step; W.queue = d_queue;
    W.gp_prog = d_gp_prog; W.gp_pc = d_gp_pc; W.gp_acc = d_gp_acc; W.gp_k = d_gp_k;
    w->finalized = true;
    w->flats.clear();
    w->flats.shrink_to_fit();
    w->builds.clear();
    w->builds.shrink_to_fit();
    // default launch shapes: the narrowest group that holds the largest scene, per size class
    if (w->max_points > 64 * 32) return fail(NPX_ERANGE, "scene too large");
    int rc2;
    npx::LaunchCfg c = clamp_cfg(w, default_shape(w->max_points), &rc2);
    if (rc2) return rc2;
    w->cfg = c;
    w->order_host = order;
    if (int rc3 = build_classes(w, true)) return rc3;
    // construction pose, at rest
    std::vector<float> zero(3 * (size_t)S, 0.f), quat(4 * (size_t)S, 0.f);
    for (int s = 0; s < S; ++s) quat[4 * s] = 1.f;
    return npx_state_set(w, zero.data(), quat.data(), zero.data(), zero.data(), nullptr);
}

int npx_state_set(npx_world *w, const float *origin, const float *quat, const float *vel,
                  const float *omega, const float *theta) {
    if (w) { ++w->state_gen; w->sg.scache_ok = false; }
    if (int rc = check_ready(w)) return rc;
    if (!origin || !quat || !vel || !omega) return fail(NPX_EINVAL, "null state array");
    CUDA_TRY(cudaSetDevice(w->device));
    const size_t S = w->S;
    float *d = w->d_stage;
    CUDA_TRY(cudaMemcpyAsync(d, origin, 3 * S * sizeof(float), cudaMemcpyHostToDevice, w->stream));
    CUDA_TRY(cudaMemcpyAsync(d + 3 * S, quat, 4 * S * sizeof(float), cudaMemcpyHostToDevice, w->stream));
    CUDA_TRY(cudaMemcpyAsync(d + 7 * S, vel, 3 * S * sizeof(float), cudaMemcpyHostToDevice, w->stream));
    CUDA_TRY(cudaMemcpyAsync(d + 10 * S, omega, 3 * S * sizeof(float), cudaMemcpyHostToDevice, w->stream));
    if (theta && w->J > 0)
        CUDA_TRY(cudaMemcpyAsync(w->W.theta, theta, w->J * sizeof(float), cudaMemcpyHostToDevice, w->stream));
    CUDA_TRY(npx::launch_init(w->W, d, d + 3 * S, d + 7 * S, d + 10 * S, w->stream));
    CUDA_TRY(cudaStreamSynchronize(w->stream));
    w->derived_stale = false;   // the set-up writes them
    return NPX_OK;
}

int npx_state_write(npx_world *w, const float *cog, const float *quat, const float *vel,
                    const float *angmom, const float *theta, const uint8_t *contact_prev,
                    int64_t step) {
    if (w) { ++w->state_gen; w->sg.scache_ok = false; }
    if (int rc = check_ready(w)) return rc;
    if (!cog || !quat || !vel || !angmom) return fail(NPX_EINVAL, "null state array");
    if (step < 0) return fail(NPX_EINVAL, "step must be >= 0");
    CUDA_TRY(cudaSetDevice(w->device));
    const size_t S = w->S;
    // the caller's arrays go to the device as they are (one copy each, all copies first); kernels
    // transpose and permute them there.  The call returns once the copies are done (the caller's
    // arrays have been read); the kernels run on, and the angular velocity and sensors are
    // recomputed when first needed.
    float *d = w->d_stage;
    const long long st64 = step;
    CUDA_TRY(cudaMemcpyAsync(d, cog, 3 * S * sizeof(float), cudaMemcpyHostToDevice, w->stream));
    CUDA_TRY(cudaMemcpyAsync(d + 3 * S, quat, 4 * S * sizeof(float), cudaMemcpyHostToDevice, w->stream));
    CUDA_TRY(cudaMemcpyAsync(d + 7 * S, vel, 3 * S * sizeof(float), cudaMemcpyHostToDevice, w->stream));
    CUDA_TRY(cudaMemcpyAsync(d + 10 * S, angmom, 3 * S * sizeof(float), cudaMemcpyHostToDevice, w->stream));
    if (theta && w->J > 0)
        CUDA_TRY(cudaMemcpyAsync(w->W.theta, theta, w->J * sizeof(float), cudaMemcpyHostToDevice, w->stream));
    if (contact_prev) CUDA_TRY(cudaMemcpyAsync(w->d_kstage, contact_prev, w->P, cudaMemcpyHostToDevice, w->stream));
    CUDA_TRY(cudaMemcpyAsync(w->d_step, &st64, sizeof st64, cudaMemcpyHostToDevice, w->stream));
    if (!w->ev_copied) CUDA_TRY(cudaEventCreateWithFlags(&w->ev_copied, cudaEventDisableTiming));
    CUDA_TRY(cudaEventRecord(w->ev_copied, w->stream));
    CUDA_TRY(npx::launch_scatter_state(w->W, d, w->stream));
    if (contact_prev)
        CUDA_TRY(npx::launch_permute_kappa(w->W.kappa, w->d_kstage, w->d_perm, w->P, true, w->stream));
    else
        CUDA_TRY(cudaMemsetAsync(w->W.kappa, 0, w->P, w->stream));
    CUDA_TRY(cudaMemsetAsync(w->W.status, 0, S * sizeof(uint32_t), w->stream));
    w->derived_stale = true;
    CUDA_TRY(cudaEventSynchronize(w->ev_copied));
    w->step = step;
    return NPX_OK;
}

int npx_contacts_read(npx_world *w, uint8_t *contact, size_t n) {
    if (int rc = check_ready(w)) return rc;
    if (!contact || n < (size_t)w->P) return fail(NPX_EINVAL, "buffer holds %zu flags, world has %d points", n, w->P);
    CUDA_TRY(cudaSetDevice(w->device));
    CUDA_TRY(npx::launch_permute_kappa(w->d_kstage, w->W.kappa, w->d_perm, w->P, false, w->stream));
    CUDA_TRY(cudaMemcpyAsync(contact, w->d_kstage, w->P, cudaMemcpyDeviceToHost, w->stream));
    CUDA_TRY(cudaStreamSynchronize(w->stream));
    return NPX_OK;
}

int npx_actuator_set(npx_world *w, int mode, const float *params) {
    if (int rc = check_ready(w)) return rc;
    if (mode != NPX_ACT_HOLD && mode != NPX_ACT_SINUSOID) return fail(NPX_EINVAL, "unknown actuator mode %d", mode);
    CUDA_TRY(cudaSetDevice(w->device));
    if (mode == NPX_ACT_SINUSOID && w->J > 0) {
        if (!params) return fail(NPX_EINVAL, "sinusoid mode needs params");
        std::vector<float4> act(w->J);
        std::vector<uint32_t> nu(w->J);
        for (int j = 0; j < w->J; ++j) {
            const float *p = params + 4 * (size_t)j;
            for (int a = 0; a < 4; ++a)
                if (!std::isfinite(p[a])) return fail(NPX_EINVAL, "joint %d: non-finite actuator parameter", j);
            act[j] = make_float4(p[0], p[1], p[2], p[3]);
            // phase increment per step in 2^-32 turns: round(f dt 2^32) modulo 2^32
            nu[j] = (uint32_t)(int64_t)std::llround((double)p[1] * (double)w->desc.dt * 4294967296.0);
        }
        CUDA_TRY(cudaMemcpyAsync((void *)w->W.act, act.data(), sizeof(float4) * w->J, cudaMemcpyHostToDevice, w->stream));
        CUDA_TRY(cudaMemcpyAsync((void *)w->W.act_nu, nu.data(), sizeof(uint32_t) * w->J, cudaMemcpyHostToDevice, w->stream));
        CUDA_TRY(cudaStreamSynchronize(w->stream));
    }
    w->act_mode = mode;
    w->W.act_mode = mode;
    clear_graphs(w);    // kernel arguments changed
    return NPX_OK;
}

int npx_gp_programs_set(npx_world *w, const uint8_t *programs) {
    if (int rc = check_ready(w)) return rc;
    if (!programs) return fail(NPX_EINVAL, "null programs");
    CUDA_TRY(cudaSetDevice(w->device));
    const size_t S = w->S;
    CUDA_TRY(cudaMemcpyAsync((void *)w->W.gp_prog, programs, 32 * S, cudaMemcpyHostToDevice, w->stream));
    CUDA_TRY(cudaMemsetAsync(w->W.gp_pc, 0, S, w->stream));
    CUDA_TRY(cudaMemsetAsync(w->W.gp_acc, 0, S, w->stream));
    CUDA_TRY(cudaMemsetAsync(w->W.gp_k, 0, std::max(w->J, 1), w->stream));
    CUDA_TRY(cudaStreamSynchronize(w->stream));
    w->act_mode = NPX_ACT_GP;
    w->W.act_mode = NPX_ACT_GP;
    clear_graphs(w);    // kernel arguments changed
    return NPX_OK;
}

int npx_gp_state_read(npx_world *w, uint8_t *pc, uint8_t *acc, int8_t *k) {
    if (int rc = check_ready(w)) return rc;
    CUDA_TRY(cudaSetDevice(w->device));
    if (pc) CUDA_TRY(cudaMemcpyAsync(pc, w->W.gp_pc, w->S, cudaMemcpyDeviceToHost, w->stream));
    if (acc) CUDA_TRY(cudaMemcpyAsync(acc, w->W.gp_acc, w->S, cudaMemcpyDeviceToHost, w->stream));
    if (k && w->J) CUDA_TRY(cudaMemcpyAsync(k, w->W.gp_k, w->J, cudaMemcpyDeviceToHost, w->stream));
    CUDA_TRY(cudaStreamSynchronize(w->stream));
    return NPX_OK;
}

int npx_gp_state_write(npx_world *w, const uint8_t *pc, const uint8_t *acc, const int8_t *k) {
    if (int rc = check_ready(w)) return rc;
    if (!pc || !acc || (!k && w->J)) return fail(NPX_EINVAL, "null controller state");
    for (int j = 0; j < w->J; ++j)
        if (k[j] < -36 || k[j] > 36) return fail(NPX_EINVAL, "joint %d: target step %d outside +-36", j, k[j]);
    CUDA_TRY(cudaSetDevice(w->device));
    CUDA_TRY(cudaMemcpyAsync(w->W.gp_pc, pc, w->S, cudaMemcpyHostToDevice, w->stream));
    CUDA_TRY(cudaMemcpyAsync(w->W.gp_acc, acc, w->S, cudaMemcpyHostToDevice, w->stream));
    if (w->J) CUDA_TRY(cudaMemcpyAsync(w->W.gp_k, k, w->J, cudaMemcpyHostToDevice, w->stream));
    CUDA_TRY(cudaStreamSynchronize(w->stream));
    return NPX_OK;
}

int npx_world_set_friction_model(npx_world *w, int flags) {
    if (int rc = check_world(w)) return rc;
    if (flags & ~(NPX_FRIC_WEIGHTED | NPX_FRIC_TILT)) return fail(NPX_EINVAL, "unknown friction flags %d", flags);
    w->W.fric_mode = flags;
    clear_graphs(w);    // kernel arguments changed
    if (w->finalized) {
        // the options select another build of the step kernel: size its launches (and raise its
        // shared-memory limit) as the current shapes' were
        CUDA_TRY(cudaSetDevice(w->device));
        int rc;
        for (auto &cls : w->classes) {
            cls.cfg = clamp_cfg_for(w, class_world(w, cls), cls.count, cls.cfg, &rc);
            if (rc) return rc;
        }
        w->cfg = clamp_cfg(w, w->cfg, &rc);
        if (rc) return rc;
    }
    return NPX_OK;
}

namespace {
// Chunks of the robot-robot broad phase, built once from the stored points: each link's points
// sorted along the longest axis of their construction-frame box and cut into chunks of at most
// `cap` points (16, doubled for a scene until it has at most 64 chunks).  Per chunk: its link,
// its construction-frame box (centre, half extent) and its points' scene-local stored indices
// (lpt, chunk-major); per scene its first chunk; per point its chunk.
int arena_tables(npx_world *w) {
    if (w->W.cbox) return NPX_OK;
    const int P = w->P, S = w->S;
    std::vector<float4> p0m(P);
    std::vector<uint8_t> plink(P), pchunk(P), clink;
    std::vector<float4> cbox;
    std::vector<int> cpo, coff(S + 1, 0);
    std::vector<uint16_t> lpt(P);
    CUDA_TRY(cudaMemcpy(p0m.data(), w->W.p0m, sizeof(float4) * (size_t)P, cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemcpy(plink.data(), w->W.plink, (size_t)P, cudaMemcpyDeviceToHost));
    int max_chunks = 1, at = 0;
    for (int s = 0; s < S; ++s) {
        const int nl = w->link_off[s + 1] - w->link_off[s], p0 = w->point_off[s];
        const int np = w->point_off[s + 1] - p0;
        std::vector<std::vector<int>> pts(nl);
        for (int i = 0; i < np; ++i) pts[plink[p0 + i]].push_back(i);
        int cap = 16, nc = 0;
        for (;;) {
            nc = 0;
            for (int l = 0; l < nl; ++l) nc += ((int)pts[l].size() + cap - 1) / cap;
            if (nc <= 64) break;
            cap *= 2;
        }
        coff[s] = (int)clink.size();
        max_chunks = std::max(max_chunks, nc);
        for (int l = 0; l < nl; ++l) {
            std::vector<int> &v = pts[l];
            const int n = (int)v.size();
            if (!n) continue;
            float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
            for (int i : v) {
                const float x[3] = {p0m[p0 + i].x, p0m[p0 + i].y, p0m[p0 + i].z};
                for (int a = 0; a < 3; ++a) { lo[a] = std::min(lo[a], x[a]); hi[a] = std::max(hi[a], x[a]); }
            }
            int ax = 0;
            for (int a = 1; a < 3; ++a)
                if (hi[a] - lo[a] > hi[ax] - lo[ax]) ax = a;
            auto coord = [&](int i) { const float4 q = p0m[p0 + i]; return ax == 0 ? q.x : ax == 1 ? q.y : q.z; };
            std::stable_sort(v.begin(), v.end(), [&](int a, int b) { return coord(a) < coord(b); });
            const int k = (n + cap - 1) / cap;
            for (int c = 0; c < k; ++c) {
                // balanced cut: chunk c holds entries [n c / k, n (c + 1) / k)
                const int b0 = (int)((long long)n * c / k), b1 = (int)((long long)n * (c + 1) / k);
                float clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
                const int local = (int)clink.size() - coff[s];
                cpo.push_back(at);
                for (int e = b0; e < b1; ++e) {
                    const int i = v[e];
                    const float x[3] = {p0m[p0 + i].x, p0m[p0 + i].y, p0m[p0 + i].z};
                    for (int a = 0; a < 3; ++a) { clo[a] = std::min(clo[a], x[a]); chi[a] = std::max(chi[a], x[a]); }
                    lpt[at++] = (uint16_t)i;
                    pchunk[p0 + i] = (uint8_t)local;
                }
                clink.push_back((uint8_t)l);
                cbox.push_back(make_float4(0.5f * (clo[0] + chi[0]), 0.5f * (clo[1] + chi[1]), 0.5f * (clo[2] + chi[2]), 0.f));
                cbox.push_back(make_float4(0.5f * (chi[0] - clo[0]), 0.5f * (chi[1] - clo[1]), 0.5f * (chi[2] - clo[2]), 0.f));
            }
        }
    }
    const int C = (int)clink.size();
    coff[S] = C;
    cpo.push_back(at);
    float4 *d_cbox;
    int *d_cpo, *d_coff;
    uint16_t *d_lpt;
    uint8_t *d_clink, *d_pchunk;
    int rc;
    if ((rc = dev_alloc(w, &d_cbox, 2 * (size_t)C)) || (rc = dev_alloc(w, &d_cpo, (size_t)C + 1)) ||
        (rc = dev_alloc(w, &d_coff, (size_t)S + 1)) || (rc = dev_alloc(w, &d_lpt, (size_t)P)) ||
        (rc = dev_alloc(w, &d_clink, (size_t)C)) || (rc = dev_alloc(w, &d_pchunk, (size_t)P)))
        return rc;
    CUDA_TRY(cudaMemcpy(d_cbox, cbox.data(), sizeof(float4) * cbox.size(), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(d_cpo, cpo.data(), sizeof(int) * cpo.size(), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(d_coff, coff.data(), sizeof(int) * coff.size(), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(d_lpt, lpt.data(), sizeof(uint16_t) * lpt.size(), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(d_clink, clink.data(), clink.size(), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(d_pchunk, pchunk.data(), pchunk.size(), cudaMemcpyHostToDevice));
    w->W.cbox = d_cbox;
    w->W.cpo = d_cpo;
    w->W.coff = d_coff;
    w->W.lpt = d_lpt;
    w->W.clink = d_clink;
    w->W.pchunk = d_pchunk;
    w->W.max_chunks = max_chunks;
    return NPX_OK;
}
}  // namespace

int npx_world_set_arenas(npx_world *w, int size, float radius) {
    if (int rc = check_ready(w)) return rc;
    const int S = w->S;
    if (size != 1 && size != 2 && size != 4) return fail(NPX_EINVAL, "arena size must be 1, 2 or 4 (got %d)", size);
    if (size > 1 && S % size) return fail(NPX_EINVAL, "%d scenes do not split into arenas of %d", S, size);
    if (size > 1 && !(radius > 0.f && std::isfinite(radius))) return fail(NPX_EINVAL, "contact radius must be > 0");
    if (size > 1 && w->max_points > 64 * (32 / size))
        return fail(NPX_ERANGE, "%d points per scene exceed the %d an arena of %d holds", w->max_points,
                    64 * (32 / size), size);
    CUDA_TRY(cudaSetDevice(w->device));
    CUDA_TRY(cudaStreamSynchronize(w->stream));   // launches in flight read the schedule
    if (size > 1) {
        if (int rc = arena_tables(w)) return rc;
        // pair lists: one per group of arenas a warp steps (at most S / size groups)
        const size_t cap = 4096, need = (size_t)(S / size + 1) * cap;
        if (w->alist_n < need) {
            uint32_t *al = nullptr;
            if (int rc = dev_alloc(w, &al, need)) return rc;
            w->W.alist = al;
            w->alist_n = need;
        }
        w->W.alist_cap = (int)cap;
    }
    auto pts = [&](int s) { return w->point_off[s + 1] - w->point_off[s]; };
    std::vector<int> order(S);
    if (size > 1) {
        // arenas whole and aligned (so that each is one warp), the one with the largest robot first
        const int na = S / size;
        std::vector<int> top(na, 0), ar(na);
        for (int a = 0; a < na; ++a)
            for (int k = 0; k < size; ++k) top[a] = std::max(top[a], pts(a * size + k));
        std::iota(ar.begin(), ar.end(), 0);
        std::stable_sort(ar.begin(), ar.end(), [&](int a, int b) { return top[a] > top[b]; });
        for (int i = 0; i < na; ++i)
            for (int k = 0; k < size; ++k) order[i * size + k] = ar[i] * size + k;
    } else {
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return pts(a) > pts(b); });
    }
    CUDA_TRY(cudaMemcpy(const_cast<int *>(w->W.order), order.data(), sizeof(int) * (size_t)S, cudaMemcpyHostToDevice));
    w->order_host = order;
    w->W.arena = size;
    w->W.rc = size > 1 ? radius : 0.f;
    clear_graphs(w);
    npx::LaunchCfg c = w->cfg;
    if (size > 1 && c.lps * size > 32) { c.lps = 32 / size; c.blocks = 0; }
    int rc;
    c = clamp_cfg(w, c, &rc);   // also raises the shared-memory limit of the kernel it selects
    if (rc) return rc;
    w->cfg = c;
    return build_classes(w, size == 1);
}

int npx_world_step(npx_world *w, int n) {
    if (int rc = check_ready(w)) return rc;
    if (n < 0) return fail(NPX_EINVAL, "n must be >= 0");
    if (n == 0) return NPX_OK;
    w->sg.scache_ok = false;   // these launches do not keep the posed-shape cache
    CUDA_TRY(cudaSetDevice(w->device));
    const int nchunks = (n + w->chunk - 1) / w->chunk;
    if (w->graphs) {
        auto it = w->graph_cache.find(n);
        if (it == w->graph_cache.end()) {
            cudaGraph_t g = nullptr;
            cudaGraphExec_t ge = nullptr;
            CUDA_TRY(cudaStreamBeginCapture(w->stream, cudaStreamCaptureModeThreadLocal));
            int rc = enqueue_steps(w, n);
            cudaError_t e = cudaStreamEndCapture(w->stream, &g);
            if (rc) { if (g) cudaGraphDestroy(g); return rc; }
            if (e != cudaSuccess) return fail(NPX_ECUDA, "graph capture: %s", cudaGetErrorString(e));
            e = cudaGraphInstantiate(&ge, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return fail(NPX_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
            if (w->graph_cache.size() >= 8) clear_graphs(w);
            it = w->graph_cache.emplace(n, ge).first;
        }
        CUDA_TRY(cudaGraphLaunch(it->second, w->stream));
    } else {
        if (int rc = enqueue_steps(w, n)) return rc;
    }
    w->launches += (long long)nchunks * (long long)w->classes.size();
    w->step += n;
    w->derived_stale = false;   // every scene's write-back rewrote them
    return NPX_OK;
}

int npx_world_sync(npx_world *w) {
    if (int rc = check_ready(w)) return rc;
    CUDA_TRY(cudaSetDevice(w->device));
    CUDA_TRY(cudaStreamSynchronize(w->stream));
    return NPX_OK;
}

int npx_sensors_read(npx_world *w, npx_sensors *o) {
    if (int rc = check_ready(w)) return rc;
    if (!o) return fail(NPX_EINVAL, "null sensors");
    CUDA_TRY(cudaSetDevice(w->device));
    if (int rc = ensure_derived(w)) return rc;
    const size_t S = w->S;
    // per-scene (AoS) blocks assembled on the device, then one copy into each caller array
    float *d = w->d_stage;
    CUDA_TRY(npx::launch_gather_state(w->W, d, w->stream));
    const struct { float *dst; size_t off, n; } parts[5] = {
        {o->cog, 0, 3 * S}, {o->quat, 3 * S, 4 * S}, {o->vel, 7 * S, 3 * S}, {o->omega, 10 * S, 3 * S},
        {o->angmom, 13 * S, 3 * S}};
    for (const auto &p : parts)
        if (p.dst) CUDA_TRY(cudaMemcpyAsync(p.dst, d + p.off, p.n * sizeof(float), cudaMemcpyDeviceToHost, w->stream));
    if (o->theta && w->J > 0) CUDA_TRY(cudaMemcpyAsync(o->theta, w->W.theta, w->J * sizeof(float), cudaMemcpyDeviceToHost, w->stream));
    if (o->contacts) CUDA_TRY(cudaMemcpyAsync(o->contacts, w->W.sensors, S * sizeof(uint32_t), cudaMemcpyDeviceToHost, w->stream));
    if (o->status) CUDA_TRY(cudaMemcpyAsync(o->status, w->W.status, S * sizeof(uint32_t), cudaMemcpyDeviceToHost, w->stream));
    CUDA_TRY(cudaStreamSynchronize(w->stream));
    if (o->step) *o->step = w->step;
    return NPX_OK;
}

int npx_points_read(npx_world *w, int scene, float *xyz, int n) {
    if (int rc = check_ready(w)) return rc;
    if (scene < 0 || scene >= w->S) return fail(NPX_EINVAL, "scene %d out of range", scene);
    const int np = w->point_off[scene + 1] - w->point_off[scene];
    if (!xyz || n < np) return fail(NPX_EINVAL, "buffer holds %d points, scene has %d", n, np);
    CUDA_TRY(cudaSetDevice(w->device));
    std::vector<float> tmp(3 * (size_t)np);
    CUDA_TRY(npx::launch_points(w->W, scene, w->d_points, w->stream));
    CUDA_TRY(cudaMemcpyAsync(tmp.data(), w->d_points, tmp.size() * sizeof(float), cudaMemcpyDeviceToHost, w->stream));
    CUDA_TRY(cudaStreamSynchronize(w->stream));
    const int p0 = w->point_off[scene];
    for (int i = 0; i < np; ++i) {
        const int u = w->perm[p0 + i] - p0;
        for (int k = 0; k < 3; ++k) xyz[3 * u + k] = tmp[3 * i + k];
    }
    return NPX_OK;
}

int npx_state_export(npx_world *w, void *blob, size_t *size) {
    if (int rc = check_ready(w)) return rc;
    if (!size) return fail(NPX_EINVAL, "null size");
    const BlobLayout b = blob_layout(w);
    if (!blob) { *size = b.end; return NPX_OK; }
    if (*size < b.end) return fail(NPX_EINVAL, "blob needs %zu bytes", b.end);
    CUDA_TRY(cudaSetDevice(w->device));
    if (int rc = ensure_derived(w)) return rc;
    char *p = static_cast<char *>(blob);
    const uint64_t hdr[8] = {kBlobMagic, (uint64_t)w->S, (uint64_t)w->P, (uint64_t)w->J,
                             (uint64_t)w->step, 0, 0, 0};
    memcpy(p, hdr, sizeof hdr);
    const size_t S = w->S;
    CUDA_TRY(cudaMemcpyAsync(p + b.st, w->W.st, sizeof(float) * npx::ST_N * S, cudaMemcpyDeviceToHost, w->stream));
    if (w->J) CUDA_TRY(cudaMemcpyAsync(p + b.theta, w->W.theta, sizeof(float) * w->J, cudaMemcpyDeviceToHost, w->stream));
    CUDA_TRY(cudaMemcpyAsync(p + b.omega, w->W.omega, sizeof(float) * 3 * S, cudaMemcpyDeviceToHost, w->stream));
    CUDA_TRY(cudaMemcpyAsync(p + b.sensors, w->W.sensors, sizeof(uint32_t) * S, cudaMemcpyDeviceToHost, w->stream));
    CUDA_TRY(cudaMemcpyAsync(p + b.status, w->W.status, sizeof(uint32_t) * S, cudaMemcpyDeviceToHost, w->stream));
    CUDA_TRY(cudaMemcpyAsync(p + b.kappa, w->W.kappa, w->P, cudaMemcpyDeviceToHost, w->stream));
    CUDA_TRY(cudaMemcpyAsync(p + b.gp_pc, w->W.gp_pc, S, cudaMemcpyDeviceToHost, w->stream));
    CUDA_TRY(cudaMemcpyAsync(p + b.gp_acc, w->W.gp_acc, S, cudaMemcpyDeviceToHost, w->stream));
    if (w->J) CUDA_TRY(cudaMemcpyAsync(p + b.gp_k, w->W.gp_k, w->J, cudaMemcpyDeviceToHost, w->stream));
    CUDA_TRY(cudaStreamSynchronize(w->stream));
    *size = b.end;
    return NPX_OK;
}

int npx_state_import(npx_world *w, const void *blob, size_t size) {
    if (w) { ++w->state_gen; w->sg.scache_ok = false; }
    if (int rc = check_ready(w)) return rc;
    const BlobLayout b = blob_layout(w);
    if (!blob || size < b.end) return fail(NPX_EINVAL, "blob too small (%zu < %zu)", size, b.end);
    uint64_t hdr[8];
    memcpy(hdr, blob, sizeof hdr);
    if (hdr[0] != kBlobMagic || hdr[1] != (uint64_t)w->S || hdr[2] != (uint64_t)w->P || hdr[3] != (uint64_t)w->J)
        return fail(NPX_EINVAL, "blob does not match this world");
    CUDA_TRY(cudaSetDevice(w->device));
    const char *p = static_cast<const char *>(blob);
    const size_t S = w->S;
    CUDA_TRY(cudaMemcpyAsync(w->W.st, p + b.st, sizeof(float) * npx::ST_N * S, cudaMemcpyHostToDevice, w->stream));
    if (w->J) CUDA_TRY(cudaMemcpyAsync(w->W.theta, p + b.theta, sizeof(float) * w->J, cudaMemcpyHostToDevice, w->stream));
    CUDA_TRY(cudaMemcpyAsync(w->W.omega, p + b.omega, sizeof(float) * 3 * S, cudaMemcpyHostToDevice, w->stream));
    CUDA_TRY(cudaMemcpyAsync(w->W.sensors, p + b.sensors, sizeof(uint32_t) * S, cudaMemcpyHostToDevice, w->stream));
    CUDA_TRY(cudaMemcpyAsync(w->W.status, p + b.status, sizeof(uint32_t) * S, cudaMemcpyHostToDevice, w->stream));
    CUDA_TRY(cudaMemcpyAsync(w->W.kappa, p + b.kappa, w->P, cudaMemcpyHostToDevice, w->stream));
    CUDA_TRY(cudaMemcpyAsync(w->W.gp_pc, p + b.gp_pc, S, cudaMemcpyHostToDevice, w->stream));
    CUDA_TRY(cudaMemcpyAsync(w->W.gp_acc, p + b.gp_acc, S, cudaMemcpyHostToDevice, w->stream));
    if (w->J) CUDA_TRY(cudaMemcpyAsync(w->W.gp_k, p + b.gp_k, w->J, cudaMemcpyHostToDevice, w->stream));
    const long long st = (long long)hdr[4];
    CUDA_TRY(cudaMemcpyAsync(w->d_step, &st, sizeof st, cudaMemcpyHostToDevice, w->stream));
    CUDA_TRY(cudaStreamSynchronize(w->stream));
    w->step = st;
    w->derived_stale = false;   // the blob's own
    return NPX_OK;
}

int npx_world_info_get(npx_world *w, npx_world_info *o) {
    if (int rc = check_ready(w)) return rc;
    if (!o) return fail(NPX_EINVAL, "null info");
    o->n_scenes = w->S; o->n_links = w->L; o->n_joints = w->J; o->n_points = w->P;
    o->max_points = w->max_points; o->max_links = w->max_links;
    o->lanes_per_scene = w->cfg.lps; o->warps_per_block = w->cfg.wpb; o->blocks = w->cfg.blocks;
    o->chunk_steps = w->chunk; o->step = w->step; o->kernel_launches = w->launches;
    o->size_classes = (int)w->classes.size();
    o->hm_window_tma = w->W.hm_tma;
    return NPX_OK;
}

int npx_world_configure(npx_world *w, int lps, int wpb, int blocks, int chunk) {
    if (int rc = check_ready(w)) return rc;
    CUDA_TRY(cudaSetDevice(w->device));
    npx::LaunchCfg c = w->cfg;
    if (lps) {
        if (lps != 4 && lps != 8 && lps != 16 && lps != 32) return fail(NPX_EINVAL, "lanes per scene must be 4, 8, 16 or 32");
        c.lps = lps;
    }
    if (wpb) {
        if (wpb < 1 || wpb > 16) return fail(NPX_EINVAL, "warps per block must be 1..16");
        c.wpb = wpb;
    }
    c.blocks = blocks > 0 ? blocks : (lps || wpb ? 0 : c.blocks);
    if (chunk < 0) return fail(NPX_EINVAL, "chunk must be >= 0");
    int rc;
    c = clamp_cfg(w, c, &rc);
    if (rc) return rc;
    if (lps || wpb || blocks) {   // an explicit shape runs the whole world in one launch
        w->cfg = c;
        if ((rc = build_classes(w, false))) return rc;
    }
    if (chunk) w->chunk = chunk;
    clear_graphs(w);
    return NPX_OK;
}

int npx_world_use_graphs(npx_world *w, int on) {
    if (int rc = check_world(w)) return rc;
    w->graphs = on != 0;
    clear_graphs(w);
    return NPX_OK;
}

int npx_surrogate_dims(npx_world *w, int *nf, int *nt) {
    if (int rc = check_ready(w)) return rc;
    if (!nf || !nt) return fail(NPX_EINVAL, "null argument");
    return surrogate_dims(w, nf, nt);
}

// Whether a surrogate window of `stride` steps may start at step n: it holds no joint-update step
// (on actuated worlds 1 <= n mod K and n mod K + stride <= K).
static bool window_fits(const npx_world *w, long long n, int stride) {
    if (w->act_mode == NPX_ACT_HOLD) return true;
    const long long K = w->desc.joint_update_steps, ph = n % K;
    return ph >= 1 && ph + stride <= K;
}

static int check_stride(const npx_world *w, int stride) {
    if (stride < 1) return fail(NPX_EINVAL, "stride must be >= 1");
    if (w->act_mode != NPX_ACT_HOLD && stride >= w->desc.joint_update_steps)
        return fail(NPX_EINVAL, "stride %d leaves no window between joint updates every %d steps", stride,
                    w->desc.joint_update_steps);
    return NPX_OK;
}

// The surrogate's shape cache (link frames, inertia, sensor points) depends on the joint angles
// alone: it stays valid over steps without a joint update and is rebuilt after one or after the
// caller writes the state.
static bool cache_valid(const npx_world *w) {
    return w->sg.cache_at == w->step && w->sg.cache_gen == w->state_gen;
}
static npx::WorldDev scache_world(const npx_world *w);

static int cache_build(npx_world *w) {
    CUDA_TRY(npx::launch_shape_cache(scache_world(w), w->sg.cache, w->stream));
    w->sg.cache_at = w->step;
    w->sg.cache_gen = w->state_gen;
    return NPX_OK;
}

// The world as the surrogate's plain launches see it: with the posed-shape cache, read at entry
// when it is current (mode 2), else written (mode 1).
static npx::WorldDev scache_world(const npx_world *w) {
    npx::WorldDev W = w->W;
    W.scache = w->sg.scache;
    W.scache_mp = w->sg.scache_mp;
    W.scache_mt = w->sg.scache_mt;
    W.scache_ml = w->sg.scache_ml;
    W.scache_mode = w->sg.scache_ok ? 2 : 1;
    return W;
}

// Makes the posed-shape cache current: a launch of zero steps over every scene rebuilds each
// shape and writes it (the state is read and written back unchanged).
static int scache_fill(npx_world *w) {
    if (w->sg.scache_ok || w->W.arena > 1) return NPX_OK;
    npx::WorldDev W = scache_world(w);
    CUDA_TRY(npx::launch_step(W, w->cfg, 0, w->stream));
    w->sg.scache_ok = true;
    w->launches += 1;
    return NPX_OK;
}

// Plain steps for every scene from the current step (reseed: their previous-step contacts from a
// detection at the current state); the shape cache follows any joint update among them.
static int plain_run(npx_world *w, int m, bool reseed) {
    const bool was_valid = cache_valid(w);
    npx::WorldDev W = scache_world(w);
    W.reseed = reseed ? 1 : 0;
    CUDA_TRY(npx::launch_step(W, w->cfg, m, w->stream));
    w->sg.scache_ok = true;   // every scene's entry written or current
    CUDA_TRY(npx::launch_advance(w->d_step, m, w->stream));
    const long long K = w->desc.joint_update_steps;
    const bool tick = w->act_mode != NPX_ACT_HOLD && (w->step + K - 1) / K * K < w->step + m;   // (step >= 0)
    w->step += m;
    w->launches += 1;
    if (tick) return cache_build(w);
    if (was_valid) w->sg.cache_at = w->step;
    return NPX_OK;
}

int npx_surrogate_collect(npx_world *w, const npx_surrogate_norm *nrm, int stride, int n_windows, float *X,
                          float *T) {
    if (int rc = check_ready(w)) return rc;
    if (w->W.arena > 1) return fail(NPX_EINVAL, "the surrogate models robots alone: not available with arenas");
    if (n_windows < 1 || !X || !T) return fail(NPX_EINVAL, "need n_windows >= 1 and X, T");
    if (int rc = check_stride(w, stride)) return rc;
    if (nrm && (!nrm->x_mu || !nrm->x_isd || !nrm->t_mu || !nrm->t_sd)) return fail(NPX_EINVAL, "incomplete norm");
    CUDA_TRY(cudaSetDevice(w->device));
    if (int rc = surrogate_buffers(w)) return rc;
    int nf, nt;
    surrogate_dims(w, &nf, &nt);
    const npx::SurCache &C = w->sg.cache;
    npx::SurrogateIO pre{nf, nt, w->max_links, w->sensor_bits};
    pre.Xraw = w->sg.F0;
    pre.cxy_out = w->sg.C0;
    if (nrm) { pre.x_mu = nrm->x_mu; pre.x_isd = nrm->x_isd; }
    npx::SurrogateIO post{nf, nt, w->max_links, w->sensor_bits};
    post.cxy_ref = w->sg.C0;
    post.prev = w->sg.F0;
    if (nrm) { post.t_mu = nrm->t_mu; post.t_sd = nrm->t_sd; }
    if (int rc = ensure_derived(w)) return rc;
    // the posed-shape cache first: the network's shape cache is built from it
    if (int rc = scache_fill(w)) return rc;
    if (!cache_valid(w))
        if (int rc = cache_build(w)) return rc;
    for (int k = 0; k < n_windows;) {
        if (!window_fits(w, w->step, stride)) {   // joint updates and what is left before them
            if (int rc = plain_run(w, 1, false)) return rc;
            continue;
        }
        pre.X = X + (size_t)k * w->S * nf;
        post.T = T + (size_t)k * w->S * nt;
        CUDA_TRY(npx::launch_features(w->W, C, pre, w->stream));
        CUDA_TRY(npx::launch_step(scache_world(w), w->cfg, stride, w->stream));
        CUDA_TRY(npx::launch_advance(w->d_step, stride, w->stream));
        CUDA_TRY(npx::launch_features(w->W, C, post, w->stream));
        w->step += stride;
        w->sg.cache_at = w->step;   // no joint update inside a window
        w->launches += 1;
        ++k;
    }
    return NPX_OK;
}

int npx_world_step_surrogate(npx_world *w, npx_mlp *net, const npx_surrogate_norm *nrm, int stride, int n_steps,
                             long long *fallbacks) {
    if (int rc = check_ready(w)) return rc;
    if (w->W.arena > 1) return fail(NPX_EINVAL, "the surrogate models robots alone: not available with arenas");
    if (!net || !nrm || !nrm->x_mu || !nrm->x_isd || !nrm->t_mu || !nrm->t_sd)
        return fail(NPX_EINVAL, "need a network and its standardisation");
    if (n_steps < 0) return fail(NPX_EINVAL, "n_steps must be >= 0");
    if (int rc = check_stride(w, stride)) return rc;
    CUDA_TRY(cudaSetDevice(w->device));
    if (int rc = surrogate_buffers(w)) return rc;
    int nf, nt, nin, nout;
    surrogate_dims(w, &nf, &nt);
    npx::mlp_dims(net, &nin, &nout);
    if (nin != nf || nout != nt) return fail(NPX_EINVAL, "network is %d -> %d, world needs %d -> %d", nin, nout, nf, nt);
    if (npx::mlp_max_batch(net) < w->sg.rows) return fail(NPX_ERANGE, "network batch capacity below %d rows", w->sg.rows);
    CUDA_TRY(cudaMemsetAsync(w->sg.total, 0, sizeof(long long), w->stream));
    cudaStream_t ns = npx::mlp_stream(net);
    int ldx = 0, ldy = 0;
    __nv_bfloat16 *Xb = npx::mlp_input(net, &ldx);
    const float *Y = npx::mlp_output(net, &ldy);
    const npx::SurCache &C = w->sg.cache;
    npx::SurrogateIO io{nf, nt, w->max_links, w->sensor_bits};
    io.Xb = Xb;
    io.ldb = ldx;
    io.x_mu = nrm->x_mu;
    io.x_isd = nrm->x_isd;
    // the plain step on the fallback list only, from contacts detected at the window's start, its
    // scenes' posed shapes read from the cache (made current below, before the first window)
    npx::WorldDev Wsub = scache_world(w);
    Wsub.scache_mode = 2;
    Wsub.order = w->sg.list;
    Wsub.sched_count = w->sg.count;
    Wsub.reseed = 1;
    // a one-step fallback list is short: one scene per warp (32 lanes) gives it the least
    // latency; longer windows take the world's own shape
    int rc_cfg = 0;
    npx::LaunchCfg fcfg = w->cfg;
    if (stride == 1 && w->max_points <= 64 * 32) {
        fcfg = clamp_cfg(w, {32, 4, 0}, &rc_cfg);
        if (rc_cfg) return rc_cfg;
    }
    if (int rc = ensure_derived(w)) return rc;
    // the posed-shape cache first: the network's shape cache is built from it
    if (int rc = scache_fill(w)) return rc;
    if (!cache_valid(w))
        if (int rc = cache_build(w)) return rc;
    // contact flags are stale after a window (the surrogate moves scenes without detecting
    // contacts): plain steps of every scene start from the contacts at the current state
    bool stale = false;
    for (int k = 0; k < n_steps;) {
        if (stride > n_steps - k || !window_fits(w, w->step, stride)) {
            // plain steps up to the next window start (or the end)
            int m = 1;
            while (k + m < n_steps && !(stride <= n_steps - k - m && window_fits(w, w->step + m, stride))) ++m;
            if (int rc = plain_run(w, m, stale)) return rc;
            stale = false;
            k += m;
            continue;
        }
        CUDA_TRY(npx::launch_features(w->W, C, io, w->stream));
        if (ns != w->stream) {
            CUDA_TRY(cudaEventRecord(w->sg.ev_w, w->stream));
            CUDA_TRY(cudaStreamWaitEvent(ns, w->sg.ev_w, 0));
        }
        if (int rc = npx::mlp_forward_packed(net, w->sg.rows)) return rc;
        if (ns != w->stream) {
            CUDA_TRY(cudaEventRecord(w->sg.ev_n, ns));
            CUDA_TRY(cudaStreamWaitEvent(w->stream, w->sg.ev_n, 0));
        }
        CUDA_TRY(npx::launch_surrogate_update(w->W, C, Y, ldy, nrm->t_mu, nrm->t_sd, w->sg.nx, w->sg.applied,
                                              w->sg.sens_new, w->sg.list, w->sg.count, w->sg.fb, w->sg.max_changed,
                                              w->stream));
        // the fallback: listed scenes kept their state; the plain step takes them through the
        // window from the contacts at that state
        CUDA_TRY(npx::launch_step(Wsub, fcfg, stride, w->stream));
        CUDA_TRY(npx::launch_accumulate(w->sg.total, w->sg.count, stride, w->stream));
        CUDA_TRY(npx::launch_advance(w->d_step, stride, w->stream));
        w->step += stride;
        w->sg.cache_at = w->step;   // no joint update inside a window
        w->launches += 1;
        stale = true;
        k += stride;
    }
    // contact flags consistent with the final state for whatever reads or steps the world next
    if (stale) CUDA_TRY(npx::launch_kappa_refresh(w->W, nullptr, nullptr, w->stream));
    if (fallbacks) {
        CUDA_TRY(cudaMemcpyAsync(fallbacks, w->sg.total, sizeof(long long), cudaMemcpyDeviceToHost, w->stream));
        CUDA_TRY(cudaStreamSynchronize(w->stream));
    }
    return NPX_OK;
}

int npx_surrogate_set_fallback(npx_world *w, int max_changed_bits) {
    if (int rc = check_ready(w)) return rc;
    if (max_changed_bits < -1) return fail(NPX_EINVAL, "max_changed_bits must be >= -1");
    w->sg.max_changed = max_changed_bits < 0 ? 32 : std::min(max_changed_bits, 32);
    return NPX_OK;
}

int npx_surrogate_fallback_counts(npx_world *w, int *counts) {
    if (int rc = check_ready(w)) return rc;
    if (!counts) return fail(NPX_EINVAL, "null counts");
    CUDA_TRY(cudaSetDevice(w->device));
    if (int rc = surrogate_buffers(w)) return rc;
    CUDA_TRY(cudaMemcpyAsync(counts, w->sg.fb, sizeof(int) * (size_t)w->S, cudaMemcpyDeviceToHost, w->stream));
    CUDA_TRY(cudaMemsetAsync(w->sg.fb, 0, sizeof(int) * (size_t)w->S, w->stream));
    CUDA_TRY(cudaStreamSynchronize(w->stream));
    return NPX_OK;
}

int npx_world_autotune(npx_world *w, int n_steps, npx_world_info *out) {
    if (int rc = check_ready(w)) return rc;
    if (n_steps < 1) return fail(NPX_EINVAL, "n_steps must be >= 1");
    CUDA_TRY(cudaSetDevice(w->device));
    CUDA_TRY(cudaStreamSynchronize(w->stream));
    // snapshot the dynamic state so the trial runs leave it untouched
    std::vector<char> blob;
    size_t bytes = 0;
    if (int rc = npx_state_export(w, nullptr, &bytes)) return rc;
    blob.resize(bytes);
    if (int rc = npx_state_export(w, blob.data(), &bytes)) return rc;
    // size classes of the schedule, each tuned on its own scenes
    if (int rc = build_classes(w, true)) return rc;
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    const int lps_list[4] = {4, 8, 16, 32};
    int rc_out = NPX_OK;
    for (auto &cls : w->classes) {
        const npx::WorldDev CW = class_world(w, cls);
        const npx::LaunchCfg saved = cls.cfg;
        npx::LaunchCfg best = saved;
        float best_ms = 1e30f;
        for (int lps : lps_list) {
            if (cls.max_points > 64 * lps) continue;
            if (w->W.arena > 1 && lps * w->W.arena > 32) continue;
            // fixed block sizes plus the "balanced" ones that spread the class's scenes evenly
            // over all SMs with 1, 2 or 3 resident blocks per SM
            std::vector<int> wpb_list = {1, 2, 4, 8, 16};
            const int G = 32 / lps;
            for (int k = 1; k <= 3; ++k) {
                const long long per = (long long)w->n_sm * G * k;
                const int wb = (int)((cls.count + per - 1) / per);
                if (wb >= 1 && wb <= 16 && std::find(wpb_list.begin(), wpb_list.end(), wb) == wpb_list.end())
                    wpb_list.push_back(wb);
            }
            for (int wpb : wpb_list) {
                int rc;
                npx::LaunchCfg c = clamp_cfg_for(w, CW, cls.count, {lps, wpb, 0}, &rc);
                if (rc) { g_err.clear(); continue; }
                float ms = 0.f;
                bool ok = true;
                for (int rep = 0; rep < 2 && ok; ++rep) {   // first run warms up
                    if (npx_state_import(w, blob.data(), bytes)) { ok = false; break; }
                    cudaEventRecord(e0, w->stream);
                    for (int done = 0; done < n_steps && ok;) {
                        const int nc = std::min(w->chunk, n_steps - done);
                        ok = npx::launch_step(CW, c, nc, w->stream) == cudaSuccess &&
                             npx::launch_advance(w->d_step, nc, w->stream) == cudaSuccess;
                        done += nc;
                    }
                    cudaEventRecord(e1, w->stream);
                    if (cudaEventSynchronize(e1) != cudaSuccess) ok = false;
                    cudaEventElapsedTime(&ms, e0, e1);
                }
                if (ok && ms < best_ms) { best_ms = ms; best = c; }
                if (!ok) {
                    rc_out = fail(NPX_ECUDA, "autotune trial lps=%d wpb=%d failed: %s", lps, wpb,
                                  cudaGetErrorString(cudaGetLastError()));
                    break;
                }
            }
            if (rc_out) break;
        }
        int rc_cfg;
        cls.cfg = clamp_cfg_for(w, CW, cls.count, rc_out ? saved : best, &rc_cfg);   // re-arms the smem limit
        if (rc_cfg && !rc_out) rc_out = rc_cfg;
        if (rc_out) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // the whole-world shape (single steps, the surrogate's fallback): that of the class of the
    // largest scenes
    if (!rc_out) {
        int rc_cfg;
        npx::LaunchCfg c = clamp_cfg(w, {w->classes[0].cfg.lps, w->classes[0].cfg.wpb, 0}, &rc_cfg);
        if (rc_cfg) rc_out = rc_cfg;
        else w->cfg = c;
        if (w->classes.size() == 1) w->classes[0].cfg = w->cfg;
        // the occupancy queries above may have lowered nothing, but the class shapes come last
        for (auto &cls : w->classes) clamp_cfg_for(w, class_world(w, cls), cls.count, cls.cfg, &rc_cfg);
    }
    clear_graphs(w);
    if (int rc = npx_state_import(w, blob.data(), bytes)) return rc;
    if (rc_out) return rc_out;
    if (out) return npx_world_info_get(w, out);
    return NPX_OK;
}

}  // extern "C"
