"""The allocation-free entry point ms2_forces_noalloc against ms2_system and
the FP64 oracle.

Callers that cannot allocate device memory (a host application that owns every
allocation and hands out a stream and buffers, a fixed memory pool or cap, a
section that must not trigger the implicit synchronisation of an allocation)
call ms2_forces_noalloc with buffers they already own.  Its working memory is
one library-owned __device__ array shared by all calls, so it must give the
same forces, torques, energy and virial as an ms2_system on the same
configuration, call after call, and agree with the oracle within the parity
tolerances.  This file is collected last on purpose.
"""
import ctypes as C
import os

import numpy as np
import pytest

from oracle import Oracle
from paper_1507_07548_gb300 import workloads as W

ms2 = pytest.importorskip("paper_1507_07548_gb300.ms2")
torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def snapshot(wl, name):
    z = np.load(os.path.join(GOLDEN, name + ".npz"))
    wl.R, wl.q, wl.v, wl.Lang = z["R"], z["q"], z["v"], z["Lang"]
    return wl


def rms_rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def reference(wl):
    s = ms2.System.from_workload(wl)
    F, tau = s.forces_torques()
    t = s.energy_terms()
    s.close()
    return F, tau, t["U_total"], t["W_total"]


def oracle(wl):
    Fo, To, to = Oracle.from_workload(wl).forces(wl.R, wl.q)
    return Fo, To, to["U_total"], to["W_total"]


def noalloc(wl, **opt):
    models, keep = ms2.make_models(wl.models)
    counts = [int((wl.species == k).sum()) for k in range(len(wl.models))]
    cnt = (C.c_int * len(counts))(*counts)
    opts = ms2.default_options(reduced=int(wl.reduced), lrc=wl.lrc, eps_rf=wl.eps_rf, **opt)
    dev = torch.device("cuda")
    R = torch.tensor(wl.R, dtype=torch.float64, device=dev)
    q = torch.tensor(wl.q, dtype=torch.float64, device=dev)
    F = torch.full((wl.N, 3), float("nan"), dtype=torch.float64, device=dev)
    tau = torch.full((wl.N, 3), float("nan"), dtype=torch.float64, device=dev)
    UW = torch.full((2,), float("nan"), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    st = ms2.lib().ms2_forces_noalloc(models, cnt, len(counts), wl.L, wl.rc, wl.elec, C.byref(opts),
                                      R.data_ptr(), q.data_ptr(), F.data_ptr(), tau.data_ptr(), UW.data_ptr(),
                                      stream or None)
    ms2.check(st)
    torch.cuda.synchronize()
    uw = UW.cpu().numpy()
    return F.cpu().numpy(), tau.cpu().numpy(), uw[0], uw[1]


def check_same(got, ref):
    F, tau, U, Wv = got
    Fr, tr, Ur, Wr = ref
    assert rms_rel(F, Fr) <= 1e-5
    if np.linalg.norm(tr) > 0:
        assert rms_rel(tau, tr) <= 1e-5
    assert abs(U - Ur) <= 1e-6 * abs(Ur)
    assert abs(Wv - Wr) <= 1e-6 * abs(Wr)


def test_noalloc_matches_system_on_consecutive_calls():
    water = snapshot(W.water_box(N=1000, rc=14.0, seed=2), "water_N1000")
    stock = snapshot(W.stockmayer_fluid(N=500, seed=4), "stockmayer_N500")
    ref_w, ref_s = reference(water), reference(stock)
    got = noalloc(water)                   # first call on the device: set-up
    check_same(got, ref_w)
    check_same(got, oracle(water))
    check_same(noalloc(water), ref_w)      # second call reuses the scratch
    got = noalloc(stock)                   # another model in the same scratch
    check_same(got, ref_s)
    check_same(got, oracle(stock))


def test_noalloc_point_lj_and_a_mixture_on_a_side_stream():
    lj = W.lj_fluid(N=256, rho=0.7, T=1.0, rc=3.5, seed=1)
    lj.R = lj.R + np.random.default_rng(3).normal(0, 0.03, lj.R.shape)   # off the lattice: F != 0
    got = noalloc(lj)                      # no electrostatics, one-site molecules
    check_same(got, reference(lj))
    check_same(got, oracle(lj))
    mix = snapshot(W.water_argon(n_water=800, n_argon=200, rc=14.0, seed=6), "water_argon_N1000")  # two models
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        got = noalloc(mix)
        again = noalloc(mix)
    check_same(got, reference(mix))
    check_same(got, oracle(mix))
    for a, b in zip(got, again):
        assert np.array_equal(a, b)


def test_noalloc_rejects_fp64():
    wl = snapshot(W.water_box(N=216, rc=9.0, seed=9), "water_N216")
    with pytest.raises(ms2.Ms2Error, match="EINVAL"):
        noalloc(wl, fp64=1)


def test_noalloc_rejects_sizes_beyond_its_maximum():
    assert ms2.lib().ms2_noalloc_scratch_bytes() < 8 << 20
    wl = W.water_box(N=4913, rc=14.0, seed=3)
    with pytest.raises(ms2.Ms2Error, match="EINVAL"):
        noalloc(wl)


def test_noalloc_call_captured_in_a_cuda_graph():
    """After a first call on the device (its set-up), a call queues only kernels
    and a device-to-device copy: it can be captured in a CUDA graph under the
    global capture mode, where allocations and pageable copies are refused, and
    every replay gives the system's forces, energy and virial."""
    wl = snapshot(W.water_box(N=216, rc=9.0, seed=9), "water_N216")
    ref = reference(wl)
    noalloc(wl)  # set-up call (scratch address, kernel attributes)
    models, keep = ms2.make_models(wl.models)
    cnt = (C.c_int * 1)(wl.N)
    opts = ms2.default_options(reduced=int(wl.reduced), lrc=wl.lrc, eps_rf=wl.eps_rf)
    dev = torch.device("cuda")
    R = torch.tensor(wl.R, dtype=torch.float64, device=dev)
    q = torch.tensor(wl.q, dtype=torch.float64, device=dev)
    F = torch.empty((wl.N, 3), dtype=torch.float64, device=dev)
    tau = torch.empty((wl.N, 3), dtype=torch.float64, device=dev)
    UW = torch.empty((2,), dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    with torch.cuda.graph(g, stream=side, capture_error_mode="global"):
        st = ms2.lib().ms2_forces_noalloc(models, cnt, 1, wl.L, wl.rc, wl.elec, C.byref(opts), R.data_ptr(),
                                          q.data_ptr(), F.data_ptr(), tau.data_ptr(), UW.data_ptr(),
                                          torch.cuda.current_stream().cuda_stream)
    ms2.check(st)
    for _ in range(2):
        F.fill_(float("nan"))
        tau.fill_(float("nan"))
        UW.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        uw = UW.cpu().numpy()
        check_same((F.cpu().numpy(), tau.cpu().numpy(), uw[0], uw[1]), ref)
