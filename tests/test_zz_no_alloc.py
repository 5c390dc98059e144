"""fricp_eval_pass_static, the entry point for callers that cannot allocate
device memory (its scratch is a static device array), checked through the C ABI
against the allocating fricp_eval_pass on two calls in a row per variant.

This file is collected last on purpose: the entry point's first call on a
device does its one-time set-up, and the test must pass both in a fresh process
and after every other test has run.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2007_07627_gb300 import synth
from tests.gpu_common import random_T

pytestmark = pytest.mark.gpu

K_SUMS = {"p2p": 17, "p2p_welsch": 17, "p2pl_welsch": 28, "p2pl": 28}


@pytest.fixture(scope="module")
def fr():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2007_07627_gb300 import build
    build.build()
    import paper_2007_07627_gb300 as fr
    fr.lib()
    return fr


def _static_pass(fr, t, p_dev, variant, Tn, nu, scale, center, stream):
    dp = ctypes.POINTER(ctypes.c_double)
    T = np.ascontiguousarray(Tn, dtype=np.float64).reshape(16)
    c = np.ascontiguousarray(center, dtype=np.float64)
    out = np.full(48, np.nan)
    st = fr.lib().fricp_eval_pass_static(t.handle, ctypes.c_void_p(p_dev.data_ptr()), int(p_dev.shape[0]),
                                         fr.VARIANTS[variant], T.ctypes.data_as(dp), float(nu), float(scale),
                                         c.ctypes.data_as(dp), ctypes.c_void_p(stream), out.ctypes.data_as(dp))
    return st, out


@pytest.mark.parametrize("variant", ["p2p", "p2p_welsch", "p2pl_welsch", "p2pl"])
def test_static_scratch_pass_matches_allocating_pass(fr, variant):
    import torch
    pair = synth.config_pair(2, 0.05)                 # M = 4000, N = 5000
    nz = oracle.normalization(pair.P.astype(float), pair.Q.astype(float))
    t = fr.target_create(pair.Q, pair.normals)
    p_dev = torch.from_numpy(pair.P).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    g = np.random.default_rng(21)
    K = K_SUMS[variant]
    for call in range(2):                             # two calls in a row share the scratch
        Tn = random_T(g, 0.3, 0.05)
        nu = 0.02 + 0.1 * g.random()
        ref = fr.eval_pass(t, p_dev, variant, Tn, nu=nu, scale=nz.s, center=nz.c)
        st, out = _static_pass(fr, t, p_dev, variant, Tn, nu, nz.s, nz.c, stream)
        assert st == 0, fr.lib().fricp_last_error()
        assert abs(out[0] - ref[0]) <= 1e-10 * max(1.0, abs(ref[0]))
        n_res = 6 if variant in ("p2pl_welsch", "p2pl") else 12
        assert np.abs(out[1:1 + n_res] - ref[1:1 + n_res]).max() <= 1e-9
        assert np.allclose(out[16:16 + K], ref[16:16 + K], rtol=1e-11, atol=1e-12 * np.abs(ref[16:16 + K]).max())


def test_static_scratch_pass_rejects_oversized_input(fr):
    import torch
    pair = synth.config_pair(1)
    t = fr.target_create(pair.Q)
    big = torch.zeros((32769, 3), dtype=torch.float32, device="cuda")
    st, _ = _static_pass(fr, t, big, "p2p", np.eye(4), 1.0, 1.0, np.zeros(3),
                         torch.cuda.current_stream().cuda_stream)
    assert st == 1
    assert b"32768" in fr.lib().fricp_last_error()


def test_static_scratch_pass_allocates_nothing(fr):
    """What the entry point exists for: after a first call (which looks up the
    scratch address and may load kernels), further calls leave the device's
    free memory and torch's allocator statistics unchanged."""
    import torch
    pair = synth.config_pair(2, 0.05)
    nz = oracle.normalization(pair.P.astype(float), pair.Q.astype(float))
    t = fr.target_create(pair.Q, pair.normals)
    p_dev = torch.from_numpy(pair.P).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    g = np.random.default_rng(22)
    for variant in ("p2p_welsch", "p2pl_welsch"):
        st, _ = _static_pass(fr, t, p_dev, variant, np.eye(4), 0.05, nz.s, nz.c, stream)
        assert st == 0, fr.lib().fricp_last_error()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    stats0 = torch.cuda.memory_stats()
    for call in range(4):
        variant = ("p2p", "p2p_welsch", "p2pl_welsch", "p2pl")[call]
        st, out = _static_pass(fr, t, p_dev, variant, random_T(g, 0.3, 0.05), 0.05, nz.s, nz.c, stream)
        assert st == 0, fr.lib().fricp_last_error()
        assert np.isfinite(out[0])
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    stats1 = torch.cuda.memory_stats()
    assert free1 == free0
    for key in ("allocation.all.allocated", "segment.all.allocated", "reserved_bytes.all.current"):
        assert stats1.get(key, 0) == stats0.get(key, 0), key


def test_static_scratch_pass_rejects_non_finite_source(fr):
    """NaN / Inf source coordinates are rejected as fricp_eval_pass rejects them,
    and the next call on good input is unaffected."""
    import torch
    pair = synth.config_pair(1)
    nz = oracle.normalization(pair.P.astype(float), pair.Q.astype(float))
    t = fr.target_create(pair.Q)
    stream = torch.cuda.current_stream().cuda_stream
    for badval in (float("nan"), float("inf")):
        P = pair.P.copy()
        P[123, 1] = badval
        st, _ = _static_pass(fr, t, torch.from_numpy(P).cuda(), "p2p", np.eye(4), 1.0, nz.s, nz.c, stream)
        assert st == 1
        assert b"NaN" in fr.lib().fricp_last_error()
    p_dev = torch.from_numpy(pair.P).cuda()
    st, out = _static_pass(fr, t, p_dev, "p2p", np.eye(4), 1.0, nz.s, nz.c, stream)
    assert st == 0
    ref = fr.eval_pass(t, p_dev, "p2p", np.eye(4), nu=1.0, scale=nz.s, center=nz.c)
    assert abs(out[0] - ref[0]) <= 1e-10 * max(1.0, abs(ref[0]))
