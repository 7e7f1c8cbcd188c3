"""The learned surrogate: its features against a numpy computation from the FP64 oracle's state,
training on simulator transitions, and rollouts with the contact-change fallback measured
against the oracle (what the trained network gains over an untrained one)."""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle.oracle import Oracle, quat_matrix
from paper_2411_05799_gb300 import npx, scenes
from tests.parity import to_gpu, quat_angle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(autouse=True)
def _own_stream():
    """Each test runs on a torch stream of its own: on the legacy default stream (handle 0) the
    library would create a stream of its own that torch's reads do not wait for."""
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        yield
    s.synchronize()


def _features_ref(o: Oracle, b, s):
    """Features of scene s from the oracle's state, written out in numpy."""
    l0, l1 = b.link_off[s], b.link_off[s + 1]
    p0, p1 = b.point_off[s], b.point_off[s + 1]
    Q, T = o.link_frames(s)
    g, Ib, M = o.mass_props(s)
    R = quat_matrix(o.q[s])
    om = o.omega()[s]
    c, v = o.c[s], o.v[s]
    f = []
    for k in range(l1 - l0):
        sel = b.plink[p0:p1] == k
        m = b.m[p0:p1][sel].astype(np.float64)
        pc = (m[:, None] * b.p0[p0:p1][sel].astype(np.float64)).sum(0) / m.sum()
        r = R @ (Q[k] @ pc + T[k] - g)
        xq = Rotation.from_matrix(Q[k]).as_quat()          # (x, y, z, w)
        ql = np.array([xq[3], *xq[:3]]) * (1 if xq[3] >= 0 else -1)
        w1, x1, y1, z1 = o.q[s]
        w2, x2, y2, z2 = ql
        qq = [w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
              w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2]
        f += [r[0], r[1], c[2] + r[2], *qq, *(v + np.cross(om, r)), *om]
    j0 = b.joint_off[s]
    for j in range(l1 - l0 - 1):
        th = o.theta[j0 + j]
        if o.n % b.joint_update_steps == 0:
            th = min(max(o.target(s, j, o.n), b.lo[l0 + j + 1]), b.hi[l0 + j + 1])
        f.append(th)
    f += [float((int(o.sensors[s]) >> k) & 1) for k in range(6)]
    return np.array(f)


@pytest.mark.parametrize("n0, stride", [(37, 1), (161, 1), (37, 20), (161, 79)])
def test_features_match_oracle_state(n0, stride):
    b = scenes.hexapod_batch(8, seed_key=31)
    o = Oracle(b)
    o.step(n0)
    w = npx.World.from_batch(b)
    to_gpu(w, o)
    nf, nt = npx.surrogate_dims(w)
    assert (nf, nt) == (271, 247)
    X = torch.zeros(8, nf, device="cuda")
    T = torch.zeros(8, nt, device="cuda")
    npx.surrogate_collect(w, 1, X.data_ptr(), T.data_ptr(), stride=stride)
    torch.cuda.synchronize()
    got = X.cpu().numpy()
    for s in range(8):
        ref = _features_ref(o, b, s)
        np.testing.assert_allclose(got[s], ref, rtol=2e-5, atol=2e-6)
    # targets: the change of the link part over the window of plain steps, against the oracle's
    # state at its end (a window of 79 steps ends just before the next joint update)
    o2 = Oracle(b)
    o2.copy_state_from(o)
    o2.step(stride)
    tg = T.cpu().numpy()
    for s in range(8):
        before = _features_ref(o, b, s)[:nt]
        after = _features_ref(o2, b, s)[:nt]
        after[0::13][:19] += o2.c[s, 0] - o.c[s, 0]     # every link relative to the first CoG
        after[1::13][:19] += o2.c[s, 1] - o.c[s, 1]
        np.testing.assert_allclose(tg[s], after - before, rtol=1e-3, atol=2e-5 * stride)


def _rollout_error(b, sur, state_world_src, n_steps, o_ref):
    """Surrogate rollout of n_steps from the oracle's state; errors of CoG and orientation."""
    w = npx.World.from_batch(b, stream=torch.cuda.current_stream().cuda_stream)
    to_gpu(w, state_world_src)
    fb = sur.step(w, n_steps)
    r = w.read()
    dc = np.linalg.norm(r["cog"] - o_ref.c, axis=1)
    da = quat_angle(r["quat"], o_ref.q)
    return dc, da, fb, r


@pytest.mark.parametrize("stride", [1, 16])
def test_training_and_50_step_rollout(stride):
    from paper_2411_05799_gb300 import surrogate
    train_b = scenes.hexapod_batch(4096, seed_key=40)
    res = surrogate.train(train_b, n_transitions=20_000_000, minibatch=8192, steps_per_chunk=16,
                          passes=2, lr=1e-3, stride=stride)
    sur = res["surrogate"]
    u = res["unexplained"]
    # held-out loss (rows the network has not been trained on) against the zero predictor's
    assert np.isfinite(u).all()
    assert u[-5:].mean() < 0.25, u[-5:]
    assert u[-5:].mean() < 0.1 * u[0], (u[0], u[-5:])
    # held-out scenes, 50 steps from a mid-gait state, against the FP64 oracle
    test_b = scenes.hexapod_batch(256, seed_key=41)
    o = Oracle(test_b, threads=8)
    o.step(1000, threads=8)
    o50 = Oracle(test_b, threads=8)
    o50.copy_state_from(o)
    o50.step(50, threads=8)
    dc, da, fb, r = _rollout_error(test_b, sur, o, 50, o50)
    assert (r["status"] == 0).all()
    assert 0 <= fb < 256 * 50 and fb % stride == 0      # whole windows fall back
    dcu, dau, fbu, ru = _rollout_error(test_b, sur.untrained_copy(), o, 50, o50)
    # what training gains: the trained network's 50-step CoG error is far below an untrained one's
    assert np.median(dc) < 0.2 * np.median(dcu), (np.median(dc), np.median(dcu))
    assert np.median(dc) < 5e-3, np.median(dc)
    assert np.median(da) < 0.2 * np.median(dau), (np.median(da), np.median(dau))


def test_posed_shape_cache_steps_bit_identically():
    """The surrogate's plain launches read each scene's posed shape from a cache instead of
    rebuilding it at entry.  Two worlds stepped alike, one whose cache is invalidated (a state
    write of its own state) before every call so that every entry is rebuilt, stay bit-identical
    over surrogate periods with fallbacks, joint updates and a one-step stride."""
    from paper_2411_05799_gb300 import surrogate
    b = scenes.hexapod_batch(256, seed_key=44)
    res = surrogate.train(scenes.hexapod_batch(512, seed_key=45), n_transitions=512 * 16 * 8,
                          minibatch=1024, steps_per_chunk=16, passes=1, stat_periods=1, warm_steps=100,
                          max_batch=256, stride=10)
    sur = res["surrogate"]
    stream = torch.cuda.current_stream().cuda_stream
    wa = npx.World.from_batch(b, stream=stream)
    wb = npx.World.from_batch(b, stream=stream)
    wa.step(41)
    wb.step(41)
    fa = fb = 0
    for n in (80, 37, 80, 3):
        fa += sur.step(wa, n)
        r = wb.read()
        wb.write_state(r["cog"], r["quat"], r["vel"], r["angmom"], r["theta"], wb.contacts(), r["step"])
        fb += sur.step(wb, n)
        ra, rb = wa.read(), wb.read()
        for k in ("cog", "quat", "vel", "angmom", "theta", "contacts", "status"):
            assert np.array_equal(ra[k], rb[k]), (n, k)
        assert np.array_equal(wa.contacts(), wb.contacts()), n
    assert fa == fb and fa > 0


def test_fallback_threshold():
    """The fallback rule: 0 (the default) falls back on any change of the contact sensors over a
    window, bit-identically to a world never told; a threshold of one bit falls back at most as
    often; -1 never falls back, keeps every state finite and ends with the sensors a detection at
    the final state gives (the world's own read-out after a rollout); -2 is refused."""
    from paper_2411_05799_gb300 import surrogate
    b = scenes.hexapod_batch(256, seed_key=46)
    res = surrogate.train(scenes.hexapod_batch(512, seed_key=47), n_transitions=512 * 16 * 8,
                          minibatch=1024, steps_per_chunk=16, passes=1, stat_periods=1, warm_steps=100,
                          max_batch=256, stride=10)
    sur = res["surrogate"]
    stream = torch.cuda.current_stream().cuda_stream
    worlds = {k: npx.World.from_batch(b, stream=stream) for k in ("default", 0, 1, -1)}
    for k, w in worlds.items():
        if k != "default":
            npx.surrogate_set_fallback(w, k)
        w.step(41)
    fb = {k: sur.step(w, 160) for k, w in worlds.items()}
    r = {k: w.read() for k, w in worlds.items()}
    for f in ("cog", "quat", "vel", "angmom", "theta", "contacts", "status"):
        assert np.array_equal(r["default"][f], r[0][f]), f
    assert fb["default"] == fb[0] > 0
    assert fb[1] <= fb[0]
    assert fb[-1] == 0
    for f in ("cog", "quat", "vel", "angmom"):
        assert np.isfinite(r[-1][f]).all(), f
    assert (r[-1]["status"] == 0).all()
    # the sensors after the rollout are the contacts at the final state: stepping on from it with
    # the plain step agrees with a world written that state
    w2 = npx.World.from_batch(b, stream=stream)
    w2.write_state(r[-1]["cog"], r[-1]["quat"], r[-1]["vel"], r[-1]["angmom"], r[-1]["theta"],
                   worlds[-1].contacts(), r[-1]["step"])
    assert np.array_equal(w2.read()["contacts"], r[-1]["contacts"])
    with pytest.raises(npx.NpxError) as e:
        npx.surrogate_set_fallback(worlds[0], -2)
    assert e.value.code == -1                              # NPX_EINVAL
