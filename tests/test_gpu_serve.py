"""Serving front end (fs_server_create / fs_submit / fs_poll / fs_server_wait),
continuous batching: requests submitted together or while a step runs share
batched steps and give, bit for bit, the result of the same request served
alone, within tolerance of fs_step; the memory in use stays within the budget;
over-budget and bad requests are refused at submit.  (The estimate test
checks fs_estimate_bytes against what a context really holds.)"""
import numpy as np
import pytest

import workloads as wl
from tests.gpu_helpers import gpu_step, make_ctx, dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1602_05650_gb300 as fs  # noqa: E402


def requests():
    out = []
    for k, (M, N, prec) in enumerate([(3, 16, fs.FS_FP64), (12, 32, fs.FS_MIXED), (1, 24, fs.FS_FP64),
                                      (20, 16, fs.FS_MIXED), (6, 32, fs.FS_FP64), (40, 24, fs.FS_MIXED)]):
        s = wl.free_space(M, N, 3.0 + M ** (1 / 3), seed=40 + k, curved_amp=0.05)
        s.f_ext = np.tile([0.1 * k, -0.2, -1.0], (s.n_points, 1))
        out.append((s, prec))
    return out


def tol_of(prec):
    return 1e-12 if prec == fs.FS_FP64 else 1e-10


def submit(sv, s, prec):
    return fs.fs_submit(sv, s.n_per_fiber, s.X, s.L, s.mu, s.eps, s.E, s.dt, f_ext=s.f_ext,
                        boundary=s.boundary, prec=prec, tol=tol_of(prec))


def served_alone(s, prec):
    """The request through a server of its own: a batch of one."""
    sv = fs.fs_server_create(4 << 30, max_slots=1)
    try:
        return fs.fs_server_wait(sv, submit(sv, s, prec), timeout_s=300)
    finally:
        fs.fs_server_destroy(sv)


def test_requests_equal_alone_and_in_the_mix():
    """Six requests of two precisions submitted at once share batched steps;
    each result equals, bit for bit, the same request served alone, and agrees
    with fs_step on the same input within its tolerance (fs_step sums a
    system's far field in another order)."""
    reqs = requests()
    sv = fs.fs_server_create(8 << 30, max_slots=8)
    tickets = [submit(sv, s, prec) for s, prec in reqs]
    res = [fs.fs_server_wait(sv, t, timeout_s=300) for t in tickets]
    st = fs.fs_server_stats(sv)
    batches = fs.fs_server_batches(sv)
    fs.fs_server_destroy(sv)
    assert st["completed"] == len(reqs)
    assert batches < len(reqs)                        # some requests shared a step
    assert max(r["info"].t_ms[7] for r in res) >= 2
    for (s, prec), r in zip(reqs, res):
        a = served_alone(s, prec)
        assert np.array_equal(r["V"], a["V"])
        assert np.array_equal(r["T"], a["T"])
        assert np.array_equal(r["X"], a["X"])
        V, T, X, _ = gpu_step(s, torch, prec=prec, tol=tol_of(prec))
        assert np.linalg.norm(r["V"] - V) <= (1e-9 if prec == fs.FS_FP64 else 1e-8) * np.linalg.norm(V)
        inf = r["info"]
        assert inf.iters > 0
        assert 0.0 <= inf.t_ms[5] <= inf.t_ms[6]


def test_requests_arriving_during_a_step_join_the_next_batch():
    """A large request occupies an engine; small ones submitted meanwhile are
    admitted together as the engines free up (fewer batches than requests),
    and each equals its result alone."""
    big = wl.free_space(256, 32, 14.0, seed=5)
    small = [wl.free_space(4 + k, 16, 4.0, seed=60 + k, curved_amp=0.05) for k in range(6)]
    sv = fs.fs_server_create(8 << 30, max_slots=16)
    t_big = submit(sv, big, fs.FS_MIXED)
    ts = [submit(sv, s, fs.FS_MIXED) for s in small]
    res = [fs.fs_server_wait(sv, t, timeout_s=300) for t in ts]
    fs.fs_server_wait(sv, t_big, timeout_s=300)
    batches = fs.fs_server_batches(sv)
    fs.fs_server_destroy(sv)
    assert batches < 1 + len(small)
    for s, r in zip(small, res):
        assert np.array_equal(r["V"], served_alone(s, fs.FS_MIXED)["V"])


def test_confined_request_equals_alone():
    s = wl.confined(12, 16, R=4.0, R_centres=2.0, n_theta=4, n_phi=8, seed=3)
    s.f_ext = np.tile([0.0, 0.0, -1.0], (s.n_points, 1))
    sv = fs.fs_server_create(4 << 30, max_slots=4)
    other = wl.free_space(5, 16, 4.0, seed=4)
    t0 = submit(sv, other, fs.FS_FP64)
    r = fs.fs_server_wait(sv, submit(sv, s, fs.FS_FP64), timeout_s=300)
    fs.fs_server_wait(sv, t0, timeout_s=300)
    fs.fs_server_destroy(sv)
    a = served_alone(s, fs.FS_FP64)
    assert np.array_equal(r["V"], a["V"]) and np.array_equal(r["T"], a["T"])
    V, T, X, _ = gpu_step(s, torch, prec=fs.FS_FP64, tol=1e-12)
    assert np.linalg.norm(r["V"] - V) <= 1e-9 * np.linalg.norm(V)


def test_budget_bounds_memory_in_use_and_rejects_oversize():
    reqs = requests()
    need = [fs.fs_estimate_bytes(s.n_per_fiber, 0, _opts(prec)) for s, prec in reqs]
    budget = int(1.05 * max(need)) + (4 << 20)
    sv = fs.fs_server_create(budget, max_slots=4)
    tickets = [submit(sv, s, prec) for s, prec in reqs]
    done = {}
    while len(done) < len(tickets):
        st = fs.fs_server_stats(sv)
        assert st["bytes_in_use"] <= budget
        for t in tickets:
            if t not in done:
                r = fs.fs_poll(sv, t)
                if r is not None:
                    done[t] = r
    big = wl.free_space(200, 32, 12.0, seed=9)
    with pytest.raises(fs.FsError) as e:
        submit(sv, big, fs.FS_MIXED)
    assert e.value.status == 7   # FS_EBUSY
    fs.fs_server_destroy(sv)
    for (s, prec), t in zip(reqs, tickets):
        assert np.array_equal(done[t]["V"], served_alone(s, prec)["V"])


def test_bad_request_is_refused_at_submit():
    """Options, physical parameters, lengths and positions are checked when
    the request is queued, so a bad request never takes a place in a batch."""
    s = wl.free_space(2, 16, 3.0, seed=6)
    sv = fs.fs_server_create(1 << 30, max_slots=1)
    try:
        for kw in ({"prec": 7}, {"tol": 2.0}):
            with pytest.raises(fs.FsError) as e:
                fs.fs_submit(sv, s.n_per_fiber, s.X, s.L, s.mu, s.eps, s.E, s.dt, f_ext=s.f_ext, **kw)
            assert e.value.status == 1             # FS_EINVAL
        with pytest.raises(fs.FsError) as e:
            fs.fs_submit(sv, s.n_per_fiber, s.X, s.L, -1.0, s.eps, s.E, s.dt)
        assert "mu > 0" in str(e.value)
        L = s.L.copy()
        L[1] = -1.0
        with pytest.raises(fs.FsError) as e:
            fs.fs_submit(sv, s.n_per_fiber, s.X, L, s.mu, s.eps, s.E, s.dt)
        assert "length" in str(e.value)
        X = s.X.copy()
        X[3, 1] = np.nan
        with pytest.raises(fs.FsError) as e:
            fs.fs_submit(sv, s.n_per_fiber, X, s.L, s.mu, s.eps, s.E, s.dt)
        assert "finite" in str(e.value)
    finally:
        fs.fs_server_destroy(sv)


def test_poll_before_done():
    s_big = wl.free_space(256, 32, 14.0, seed=5)
    sv = fs.fs_server_create(8 << 30, max_slots=1)
    t1 = submit(sv, s_big, fs.FS_MIXED)
    assert fs.fs_poll(sv, t1) is None          # the step takes longer than this call
    r = fs.fs_server_wait(sv, t1, timeout_s=300)
    assert np.all(np.isfinite(r["V"]))
    with pytest.raises(fs.FsError):
        fs.fs_poll(sv, t1)                     # the ticket was released
    fs.fs_server_destroy(sv)


def _opts(prec, restart=60):
    o = fs.fs_options_default()
    o.prec = prec
    o.restart = restart
    return o


@pytest.mark.parametrize("case", ["fp64", "mixed", "ragged", "confined"])
def test_estimate_bounds_device_bytes(case):
    if case == "confined":
        s = wl.confined(12, 16, R=4.0, R_centres=2.0, n_theta=4, n_phi=8, seed=4)
    elif case == "ragged":
        s = wl.free_space(10, [16, 24, 32, 16, 64, 8, 24, 32, 16, 48], 5.0, seed=8)
    else:
        s = wl.free_space(64, 32, 10.0, seed=8, curved_amp=0.05)
    s.f_ext = np.tile([0.0, 0.0, -1.0], (s.n_points, 1))
    prec = fs.FS_MIXED if case in ("mixed", "ragged") else fs.FS_FP64
    h = make_ctx(s, prec=prec, tol=1e-10)
    fs.fs_set_state(h, dev(s.X, torch), dev(s.L, torch), dev(s.f_ext, torch))
    fs.fs_step(h)
    used = fs.fs_device_bytes(h)
    fs.fs_destroy(h)
    ns = 0 if s.boundary is None else s.boundary.nodes.shape[0]
    est = fs.fs_estimate_bytes(s.n_per_fiber, ns, _opts(prec))
    assert used <= est
    assert est <= 2 * used + (1 << 20)
