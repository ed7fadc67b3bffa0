"""ij_step_noalloc: the allocation-free step against the handle-based step.

Callers that may not allocate device memory where they step the lattice (a
plugin whose host framework owns all device memory, a loop that must keep a
fixed memory footprint) use ij_step_noalloc with their own population
buffers.  This test calls it through the C ABI twice in a row and checks each
result against ij_step on a one-lattice handle, within the single-step parity
tolerance of the other GPU tests, and checks that a step which crosses the
lattice's velocity limit is reported through the status slot.  It runs alone
or after the other tests (it depends on nothing they leave behind).
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

WEIGHTS = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4, dtype=np.float32)


def _rel(a, b, scale):
    return float(np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64)).max() / scale)


def test_noalloc_step_matches_handle_step_twice():
    import torch
    from paper_1702_04487_gb300 import inkjet, workloads as W

    assert torch.cuda.is_available()
    p = W.small_nozzle(nx=48, ny=96)
    n0 = np.float32(0.5 * (p["rho_ink"] + p["rho_air"]))
    h = inkjet.ij_create(p)
    f_abs, g = inkjet.ij_get_state(h, 0)
    fluid = f_abs[0] != 0.0
    # stored layout: deviations from w_i n0 on fluid cells, 0 on solid cells
    dev = np.where(fluid[None], f_abs - WEIGHTS[:, None, None] * n0, 0.0).astype(np.float32)
    bufs_f = [torch.from_numpy(dev).cuda(), torch.zeros_like(torch.from_numpy(dev)).cuda()]
    bufs_g = [torch.from_numpy(g).cuda(), torch.zeros_like(torch.from_numpy(g)).cuda()]
    rec = torch.zeros(13, dtype=torch.float64, device="cuda")  # one record (ij_obs)
    status = torch.full((1,), 7, dtype=torch.int32, device="cuda")  # numeric flag slot
    params = inkjet.make_params(p)
    stream = torch.cuda.current_stream().cuda_stream

    for t in (0, 1):
        src, dst = t % 2, (t + 1) % 2
        st = inkjet._lib.ij_step_noalloc(C.byref(params), t, bufs_f[src].data_ptr(),
                                         bufs_g[src].data_ptr(), bufs_f[dst].data_ptr(),
                                         bufs_g[dst].data_ptr(), rec.data_ptr(),
                                         status.data_ptr(), C.c_void_p(stream))
        assert st == inkjet.IJ_OK, inkjet.ij_last_error()
        state_t = inkjet.ij_get_state(h, 0)
        inkjet.ij_step(h, 1)
        torch.cuda.synchronize()
        f_ref, g_ref = inkjet.ij_get_state(h, 0)
        assert int(status.item()) == 0
        f_new = bufs_f[dst].cpu().numpy()
        f_new_abs = np.where(fluid[None], f_new + WEIGHTS[:, None, None] * n0, 0.0)
        assert _rel(f_new_abs, f_ref, np.abs(f_ref).max()) < 3e-6
        assert _rel(bufs_g[dst].cpu().numpy(), g_ref, 4.5) < 3e-6
        # the record describes the state at t
        r = rec.cpu().numpy()
        assert r[0] == t
        mass_n = state_t[0].astype(np.float64).sum(0)[fluid].sum()
        assert abs(r[1] - mass_n) < 1e-6 * mass_n
        if t == 0:
            obs, _ = inkjet.ij_observe(h, 0, phi=False)
            assert obs["step"] == 0
            for key, col in (("mass_n", 1), ("mass_phi", 2), ("droplet_volume", 6),
                             ("head_y", 11), ("tail_y", 12)):
                assert abs(r[col] - obs[key]) <= 1e-6 * max(1.0, abs(obs[key]))


def test_noalloc_rejects_fp16_storage():
    """The allocation-free step takes FP32 buffers only; FP16 storage is
    refused on the host before any device work."""
    from paper_1702_04487_gb300 import inkjet, workloads as W

    p = inkjet.make_params(W.small_nozzle(precision=1))
    dummy = C.c_void_p(16)
    st = inkjet._lib.ij_step_noalloc(C.byref(p), 0, dummy, dummy, C.c_void_p(32),
                                     C.c_void_p(48), None, None, None)
    assert st == inkjet.IJ_ERR_PARAM
    assert "FP32" in inkjet.ij_last_error()


def test_noalloc_rejects_lattices_beyond_its_fixed_scratch():
    from paper_1702_04487_gb300 import inkjet, workloads as W

    p = inkjet.make_params(W.small_nozzle(nx=48, ny=9000))
    dummy = C.c_void_p(16)
    st = inkjet._lib.ij_step_noalloc(C.byref(p), 0, dummy, dummy, C.c_void_p(32),
                                     C.c_void_p(48), None, None, None)
    assert st == inkjet.IJ_ERR_PARAM
    assert "8192" in inkjet.ij_last_error()


def test_noalloc_reports_a_step_past_the_velocity_limit():
    """A state whose flow exceeds |u| = 0.3 in part of the lattice: the step
    kernel flags it (and stops writing that lattice), and the call hands the
    flag to the caller through status_out, so the partly written output is
    not taken for a result.  The next call on a sound state reports 0."""
    import torch
    from paper_1702_04487_gb300 import inkjet, workloads as W

    p = W.small_nozzle(nx=48, ny=96)
    n0 = np.float32(0.5 * (p["rho_ink"] + p["rho_air"]))
    h = inkjet.ij_create(p)
    f_abs, g = inkjet.ij_get_state(h, 0)
    fluid = f_abs[0] != 0.0
    dev = np.where(fluid[None], f_abs - WEIGHTS[:, None, None] * n0, 0.0).astype(np.float32)
    fast = dev.copy()
    n = f_abs.sum(0)
    # rows 70..79: momentum n u_y with u_y = 0.4 carried by f_2 - f_4
    fast[2, 70:80] += np.where(fluid[70:80], 0.2 * n[70:80], 0.0)
    fast[4, 70:80] -= np.where(fluid[70:80], 0.2 * n[70:80], 0.0)
    params = inkjet.make_params(p)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    g_in = torch.from_numpy(g).cuda()
    f_out = torch.zeros(dev.shape, dtype=torch.float32, device="cuda")
    g_out = torch.zeros(g.shape, dtype=torch.float32, device="cuda")
    for state, flagged in ((fast, True), (dev, False)):
        f_in = torch.from_numpy(state).cuda()
        st = inkjet._lib.ij_step_noalloc(C.byref(params), 0, f_in.data_ptr(), g_in.data_ptr(),
                                         f_out.data_ptr(), g_out.data_ptr(), None,
                                         status.data_ptr(), stream)
        assert st == inkjet.IJ_OK, inkjet.ij_last_error()
        torch.cuda.synchronize()
        assert (int(status.item()) != 0) == flagged
