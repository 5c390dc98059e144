"""Serving loop (fricp_server_*) through the C ABI: continuous batching.

Requests arrive while others are on the GPU, wait in the queue for a slot and
for room in the HBM budget, and are advanced together. Each served result must
equal, bit for bit, the result of fricp_register on the same request alone.
"""
import numpy as np
import pytest

from paper_2007_07627_gb300 import synth

pytestmark = pytest.mark.gpu

COUNTERS = ("status", "iterations", "corr_passes", "aa_accepted", "reverts", "line_search_trials", "stages",
            "device_steps", "nu_max", "nu_min", "final_energy")


@pytest.fixture(scope="module")
def fr():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2007_07627_gb300 import build
    build.build()
    import paper_2007_07627_gb300 as fr
    fr.lib()
    return fr


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


def _same(a, b, what):
    for k in COUNTERS:
        assert a[k] == b[k], (what, k, a[k], b[k])
    assert np.array_equal(a["R"], b["R"]) and np.array_equal(a["t"], b["t"]), what


def _serve_all(fr, srv, reqs, targets, arrivals, on_device=False, nsteps=8):
    """Submit request k once `arrivals[k]` server steps have run; step until all finish."""
    tickets, results, tick = {}, {}, 0
    srcs = [_dev(p.P) if on_device else p.P for _, p in reqs]
    max_in_flight = 0
    while len(results) < len(reqs):
        for k in range(len(reqs)):
            if k not in tickets and arrivals[k] <= tick:
                v, p = reqs[k]
                tickets[k] = srv.submit(targets[k], srcs[k], fr.params_default(v))
        inf, q = srv.step(nsteps)
        max_in_flight = max(max_in_flight, inf)
        tick += 1
        for k, t in tickets.items():
            if k not in results:
                r = srv.poll(t)
                if r is not None:
                    results[k] = r
        assert tick < 100000
    return results, max_in_flight


@pytest.mark.parametrize("on_device", [False, True])
def test_served_equals_alone_with_queueing(fr, on_device):
    reqs = synth.serve_requests(seed=777, n=10, lo=300, hi=5000)
    targets = [fr.target_create(p.Q, p.normals) for _, p in reqs]
    srv = fr.Server(hbm_budget=64 << 20, max_slots=3, steps_per_sync=8)
    arrivals = [0, 0, 0, 0, 2, 3, 3, 7, 12, 20]
    results, max_inf = _serve_all(fr, srv, reqs, targets, arrivals, on_device)
    assert max_inf <= 3
    for k, (v, p) in enumerate(reqs):
        alone = fr.register(targets[k], p.P, params=fr.params_default(v))
        _same(results[k], alone, f"request {k} ({v}, M={p.M}, N={p.N})")
    srv.destroy()
    for t in targets:
        t.destroy()


def test_budget_limits_admission(fr):
    reqs = synth.serve_requests(seed=778, n=6, lo=3000, hi=3000)
    assert all(p.M == 3000 for _, p in reqs)
    targets = [fr.target_create(p.Q, p.normals) for _, p in reqs]
    # one request holds 28 B per point and 224 B per 256 points (87 KB for 3000
    # points) plus one state (under 5 KB), and its target's index 32 B per point
    # with normals and 64 B per bucket of 16 (112 KB for 3000 points): every
    # request has its own target, so 300 KB admits one request at a time
    srv = fr.Server(hbm_budget=300_000, max_slots=16, steps_per_sync=4)
    results, max_inf = _serve_all(fr, srv, reqs, targets, [0] * len(reqs), nsteps=4)
    assert max_inf == 1
    for k, (v, p) in enumerate(reqs):
        _same(results[k], fr.register(targets[k], p.P, params=fr.params_default(v)), f"request {k}")
    srv.destroy()
    for t in targets:
        t.destroy()


def test_queue_full_oversize_and_unknown_ticket(fr):
    pair = synth.config_pair(1, 0.5)
    t = fr.target_create(pair.Q)
    srv = fr.Server(hbm_budget=1 << 20, max_slots=2, max_queue=2)
    prm = fr.params_default("p2p_welsch")
    a = srv.submit(t, pair.P, prm)
    srv.submit(t, pair.P, prm)
    with pytest.raises(fr.FricpError) as ei:
        srv.submit(t, pair.P, prm)
    assert "EBUSY" in str(ei.value)
    big = np.zeros((1 << 16, 3), np.float32)
    srv2 = fr.Server(hbm_budget=1 << 20, max_slots=2)
    with pytest.raises(fr.FricpError) as ei:
        srv2.submit(t, big, prm)
    assert "budget" in str(ei.value)
    with pytest.raises(fr.FricpError):
        srv.poll(a + 100)
    while srv.poll(a) is None:
        srv.step(16)
    srv.destroy()
    srv2.destroy()
    t.destroy()


def test_bad_request_fails_alone(fr):
    import torch
    reqs = synth.serve_requests(seed=779, n=3, lo=500, hi=1500)
    targets = [fr.target_create(p.Q, p.normals) for _, p in reqs]
    srv = fr.Server(max_slots=4)
    bad = _dev(reqs[1][1].P)
    bad[3, 1] = float("nan")                      # found on the device at admission
    tickets = [srv.submit(targets[0], reqs[0][1].P, fr.params_default(reqs[0][0])),
               srv.submit(targets[1], bad, fr.params_default(reqs[1][0])),
               srv.submit(targets[2], reqs[2][1].P, fr.params_default(reqs[2][0]))]
    torch.cuda.synchronize()
    res = {}
    while len(res) < 3:
        srv.step(16)
        for k, tk in enumerate(tickets):
            if k not in res:
                r = srv.poll(tk)
                if r is not None:
                    res[k] = r
    assert res[1]["status"] == "EINVAL"
    for k in (0, 2):
        v, p = reqs[k]
        _same(res[k], fr.register(targets[k], p.P, params=fr.params_default(v)), f"request {k}")
    srv.destroy()
    for t in targets:
        t.destroy()
