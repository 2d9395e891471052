"""The continuous-batching server: remap and particle requests over resident
meshes, results identical alone and in a mix of concurrent requests,
admission by device memory, host-side timeouts and cancellation."""
import threading

import numpy as np
import pytest

from paper_2501_12349_b300 import workloads as W
from parity_util import compare_eval, compare_find, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    return t


@pytest.fixture(scope="module")
def fp():
    import paper_2501_12349_b300 as f
    f.lib()
    return f


@pytest.fixture(scope="module")
def resident(fp, torch):
    rng = np.random.default_rng(50)
    out = []
    for n, p, A in ((6, 3, 0.2), (5, 4, 0.3), (4, 5, 0.1)):
        coords = W.hex_mesh(n, p, A)
        fld, _ = W.polynomial_field(coords, rng, 3)
        vel = W.velocity_field(coords)
        m = fp.Mesh(torch.from_numpy(coords).cuda(), 3, 3, p)
        out.append((m, torch.from_numpy(fld).cuda(), torch.from_numpy(vel).cuda(), 1.0 / n))
    yield out
    for e in out:
        e[0].close()


def server_of(fp, resident, **kw):
    return fp.Server([(m, f, v) for m, f, v, h in resident], **kw)


def reference_particles(fp, torch, mesh, vel, x0, steps, dt):
    """Explicit midpoint steps with the single-mesh GPU find + eval calls."""
    x = torch.from_numpy(x0.copy()).cuda()
    for _ in range(steps):
        c, e, r, d2 = mesh.find(x)
        u = mesh.eval(c, e, r, vel)
        xm = x + 0.5 * dt * u.T
        c, e, r, d2 = mesh.find(xm.contiguous())
        u = mesh.eval(c, e, r, vel)
        x = x + dt * u.T
    return to_np(x), tuple(to_np(t) for t in mesh.find(x.contiguous()))


def test_remap_matches_find_eval(fp, torch, resident):
    s = server_of(fp, resident)
    rng = np.random.default_rng(51)
    pts = rng.uniform(-0.02, 1.02, (5000, 3))
    rid = s.submit(0, fp.FP_REQ_REMAP, pts)
    code, elem, r, d2, u = s.wait(rid)
    m, fld, vel, h = resident[0]
    m.set_precision(fp.FP_MIXED)
    ref = m.find(torch.from_numpy(pts).cuda())
    uref = to_np(m.eval(*ref[:3], fld))
    m.set_precision(fp.FP_F64)
    ref = tuple(to_np(t) for t in ref)
    compare_find(ref, (code, elem, r, d2), label="server remap")
    assert np.array_equal(ref[0], code) and np.array_equal(ref[1], elem)
    compare_eval(to_np(fld), m.NE, m.N ** 3, elem, uref, u, "server remap eval")
    s.close()


def test_particles_match_reference(fp, torch, resident):
    s = server_of(fp, resident, precision=fp.FP_F64)
    rng = np.random.default_rng(52)
    x0 = rng.uniform(0.02, 0.98, (2000, 3))
    m, fld, vel, h = resident[1]
    dt = 0.1 * h / np.sqrt(2.01)
    rid = s.submit(1, fp.FP_REQ_PARTICLE, x0, rk_steps=4, dt=dt)
    code, elem, r, d2, x = s.wait(rid)
    xr, (rc, re, rr, rd) = reference_particles(fp, torch, m, vel, x0, 4, dt)
    assert np.max(np.abs(x - xr)) < 1e-10
    assert np.array_equal(code, rc) and np.array_equal(elem, re)
    assert np.max(np.abs(r - rr)) < 1e-10
    assert np.max(np.abs(x - x0)) > 0.1 * dt  # the particles moved
    s.close()


@pytest.mark.parametrize("precision", ["mixed", "f64"])
def test_same_alone_and_in_mix(fp, torch, resident, precision):
    """A request's results do not depend on what else is in flight: the
    meshes' element shapes of one tick run side by side on forked streams,
    in either precision."""
    rng = np.random.default_rng(53)
    pa = rng.uniform(-0.02, 1.02, (3000, 3))
    pp = rng.uniform(0.05, 0.95, (2000, 3))
    dt = 0.02
    s = server_of(fp, resident, precision=fp.FP_MIXED if precision == "mixed" else fp.FP_F64)
    alone_a = [a.copy() for a in s.wait(s.submit(2, fp.FP_REQ_REMAP, pa))]
    alone_p = [a.copy() for a in s.wait(s.submit(0, fp.FP_REQ_PARTICLE, pp, rk_steps=3, dt=dt))]
    ids = []
    for k in range(40):
        mesh = int(rng.integers(0, 3))
        n = int(np.exp(rng.uniform(np.log(100), np.log(20000))))
        if k % 2:
            ids.append(s.submit(mesh, fp.FP_REQ_REMAP, rng.uniform(-0.02, 1.02, (n, 3))))
        else:
            ids.append(s.submit(mesh, fp.FP_REQ_PARTICLE, rng.uniform(0.05, 0.95, (n, 3)), rk_steps=2, dt=dt))
        if k == 10:
            ra = s.submit(2, fp.FP_REQ_REMAP, pa)
        if k == 20:
            rp = s.submit(0, fp.FP_REQ_PARTICLE, pp, rk_steps=3, dt=dt)
    mix_a = s.wait(ra)
    mix_p = s.wait(rp)
    for i in ids:
        s.wait(i)
    st = s.stats()
    assert st.completed == 44 and st.active == 0 and st.bytes_in_use == 0
    assert st.ticks < 44 * 5  # stages of different requests shared ticks
    for a, b in zip(alone_a, mix_a):
        assert np.array_equal(a, b)
    for a, b in zip(alone_p, mix_p):
        assert np.array_equal(a, b)
    s.close()


def test_admission_by_memory(fp, torch, resident):
    budget = 4 << 20
    s = server_of(fp, resident, mem_budget=budget)
    rng = np.random.default_rng(54)
    with pytest.raises(fp.FindptsError) as err:
        s.submit(0, fp.FP_REQ_REMAP, rng.uniform(0, 1, (200000, 3)))  # can never fit
    assert err.value.status == fp.FP_ENOMEM
    peak = [0]
    stop = threading.Event()

    def watch():
        while not stop.is_set():
            peak[0] = max(peak[0], s.stats().bytes_in_use)

    th = threading.Thread(target=watch)
    th.start()
    ids = [s.submit(i % 3, fp.FP_REQ_REMAP, rng.uniform(0, 1, (20000, 3))) for i in range(12)]
    for i in ids:
        s.wait(i)
    stop.set()
    th.join()
    assert 0 < peak[0] <= budget
    assert s.stats().completed == 12
    s.close()


def test_wait_timeout_and_cancel(fp, torch, resident):
    s = server_of(fp, resident, max_active=1)
    rng = np.random.default_rng(55)
    big = s.submit(0, fp.FP_REQ_PARTICLE, rng.uniform(0.05, 0.95, (200000, 3)), rk_steps=20, dt=0.001)
    small = s.submit(1, fp.FP_REQ_REMAP, rng.uniform(0, 1, (100, 3)))
    with pytest.raises(fp.FindptsError) as err:
        s.wait(small, timeout_s=1e-4)
    assert err.value.status == fp.FP_ETIMEDOUT
    rc = s.cancel(small)
    if rc == 0:
        assert s.poll(small) == (True, fp.FP_ECANCELED)
    s.wait(big, timeout_s=120)
    assert s.stats().timeouts == 0
    s.close()


def test_tiles_small_ticks(fp, torch, resident):
    """With a point budget of 1000 per tick every stage is split into many
    tiles (tile-level interleaving): results equal those of the default
    budget, and a small request submitted after a large one finishes first."""
    rng = np.random.default_rng(56)
    pa = rng.uniform(-0.02, 1.02, (30000, 3))
    pp = rng.uniform(0.05, 0.95, (8000, 3))
    s0 = server_of(fp, resident)
    ref_a = [a.copy() for a in s0.wait(s0.submit(1, fp.FP_REQ_REMAP, pa))]
    ref_p = [a.copy() for a in s0.wait(s0.submit(2, fp.FP_REQ_PARTICLE, pp, rk_steps=2, dt=0.01))]
    s0.close()
    s = server_of(fp, resident, tick_points=1000)
    big = s.submit(0, fp.FP_REQ_PARTICLE, rng.uniform(0.05, 0.95, (200000, 3)), rk_steps=4, dt=0.001)
    small = s.submit(1, fp.FP_REQ_REMAP, rng.uniform(0, 1, (200, 3)))
    s.wait(small, timeout_s=60)
    done_big, _ = s.poll(big)
    assert not done_big  # the small request passed the large one
    got_a = s.wait(s.submit(1, fp.FP_REQ_REMAP, pa))
    got_p = s.wait(s.submit(2, fp.FP_REQ_PARTICLE, pp, rk_steps=2, dt=0.01))
    for a, b in zip(ref_a, got_a):
        assert np.array_equal(a, b)
    for a, b in zip(ref_p, got_p):
        assert np.array_equal(a, b)
    s.wait(big, timeout_s=120)
    assert s.stats().ticks > 60
    s.close()


def test_tick_watchdog(fp, torch, resident):
    """A tick past the watchdog limit fails its requests with FP_ETIMEDOUT on
    the host (the kernels themselves finish normally; no GPU fault is
    involved), the request memory is released once the tick has ended, and
    the server keeps serving with a normal limit afterwards."""
    import time
    s = server_of(fp, resident, tick_timeout_s=1e-7)
    rng = np.random.default_rng(57)
    rid = s.submit(0, fp.FP_REQ_PARTICLE, rng.uniform(0.05, 0.95, (200000, 3)), rk_steps=2, dt=0.001)
    with pytest.raises(fp.FindptsError) as err:
        s.wait(rid, timeout_s=60)
    assert err.value.status == fp.FP_ETIMEDOUT
    st = s.stats()
    assert st.timeouts >= 1
    deadline = time.time() + 30
    while s.stats().bytes_in_use != 0 and time.time() < deadline:
        time.sleep(0.01)
    assert s.stats().bytes_in_use == 0 and s.stats().active == 0
    s.close()
    s2 = server_of(fp, resident)
    code, elem, r, d2, u = s2.wait(s2.submit(0, fp.FP_REQ_REMAP, rng.uniform(0, 1, (1000, 3))))
    assert np.all(code != 2)
    s2.close()


@pytest.fixture(scope="module")
def config5_scale():
    """One resident mesh as config 5 serves them at its highest order:
    27^3 = 19,683 hexes of order 7 (512 nodes each), a smooth deformation of
    amplitude 0.25, a random degree-3 polynomial to remap and the nodal
    velocity field of the particle requests, with the oracle's mesh."""
    import oracle
    coords = W.hex_mesh(27, 7, 0.25)
    rng = np.random.default_rng(58)
    fld, _ = W.polynomial_field(coords, rng, 3)
    vel = W.velocity_field(coords)
    return coords, fld, vel, oracle.OracleMesh(coords, 3, 3, 8)


def oracle_particles(om, vel, x0, steps, dt):
    """Explicit midpoint steps (the RK2 of Sec. 6.7's particle tracking)
    driven by the oracle: find + eval of the nodal velocity at x, then at
    the midpoint, advanced with numpy; returns the final positions and the
    oracle's find there."""
    x = x0.copy()
    for _ in range(steps):
        o = om.findpts(x)
        xm = x + 0.5 * dt * om.eval(vel, *o[:3]).T
        o = om.findpts(xm)
        x = x + dt * om.eval(vel, *o[:3]).T
    return x, om.findpts(x)


@pytest.mark.parametrize("precision", ["mixed", "f64"])
def test_server_matches_oracle_config5_scale(fp, torch, config5_scale, precision):
    """Served requests on a config-5-sized mesh of order 7 against the
    oracle: a remap request (20,000 points, 5% outside the domain) must
    match the oracle's find + eval, and a 4-step particle request (5,000
    particles, dt = 0.1 h / |u|max) must match the oracle-driven midpoint
    rule: code and element exact, r within 1e-10, positions within 1e-10."""
    coords, fld, vel, om = config5_scale
    m = fp.Mesh(torch.from_numpy(coords).cuda(), 3, 3, 7)
    s = fp.Server([(m, torch.from_numpy(fld).cuda(), torch.from_numpy(vel).cuda())],
                  precision=fp.FP_MIXED if precision == "mixed" else fp.FP_F64)
    rng = np.random.default_rng(59)
    pts = rng.uniform(-0.017, 1.017, (20000, 3))
    xp = rng.uniform(0.02, 0.98, (5000, 3))
    dt = 0.1 * (1.0 / 27) / np.sqrt(1.01)
    ra = s.submit(0, fp.FP_REQ_REMAP, pts)
    rp = s.submit(0, fp.FP_REQ_PARTICLE, xp, rk_steps=4, dt=dt)
    code, elem, r, d2, u = s.wait(ra, timeout_s=120)
    o = om.findpts(pts)
    res = compare_find(o, (code, elem, r, d2), label=f"served remap {precision}")
    assert min(res["codes"]) > 0
    compare_eval(fld, om.NE, 8 ** 3, o[1], om.eval(fld, *o[:3]), u, f"served remap eval {precision}")
    pc, pe, pr, pd, x = s.wait(rp, timeout_s=120)
    xo, oo = oracle_particles(om, vel, xp, 4, dt)
    assert np.max(np.abs(x - xo)) < 1e-10
    assert np.max(np.abs(x - xp)) > 0.3 * dt  # the particles moved
    compare_find(oo, (pc, pe, pr, pd), label=f"served particles {precision}")
    s.close()
    m.close()


def test_policies_same_results(fp, torch, resident):
    """The tick policy (least slack, the default, or least work left in the
    stage) changes only the order in which tiles are served: results are
    identical; an unknown policy or a negative slack factor is refused."""
    rng = np.random.default_rng(60)
    pa = rng.uniform(-0.02, 1.02, (20000, 3))
    pp = rng.uniform(0.05, 0.95, (6000, 3))
    got = []
    for pol in (fp.FP_SCHED_SLACK, fp.FP_SCHED_SRPT):
        s = server_of(fp, resident, policy=pol, tick_points=4096)
        ids = [s.submit(1, fp.FP_REQ_REMAP, pa), s.submit(2, fp.FP_REQ_PARTICLE, pp, rk_steps=2, dt=0.01)]
        ids += [s.submit(k % 3, fp.FP_REQ_REMAP, rng.uniform(0, 1, (300, 3))) for k in range(6)]
        got.append([[a.copy() for a in s.wait(i)] for i in ids[:2]])
        for i in ids[2:]:
            s.wait(i)
        s.close()
    for a, b in zip(got[0], got[1]):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
    for kw in ({"policy": 7}, {"slack_factor": -1.0}):
        with pytest.raises(fp.FindptsError) as err:
            server_of(fp, resident, **kw)
        assert err.value.status == fp.FP_EINVAL
