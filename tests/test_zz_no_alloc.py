"""chem_step_noalloc, the allocation-free single step, against the context path.

Some callers cannot let a library allocate device memory (code running under another
framework's memory pool that owns the device, real-time loops that must not allocate,
hosts whose allocator must not be re-entered). For them chem_step_noalloc takes one FP64
step of species held in the caller's own device buffers, with its working memory in a
fixed array inside the library. This test owns every buffer (torch tensors), calls the
entry point through the C ABI twice in a row, feeding the first call's output to the
second, and checks each result against chem_init + chem_run_until advanced by the same
steps: identical ids, types and events, positions within 1e-12 L.

The file is named so that pytest collects it last."""
import ctypes

import numpy as np
import pytest

from harness import cuda_available, event_matrix
from paper_2509_03313_gb300 import chem, workloads as W

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not cuda_available(), reason="needs a CUDA GPU")]


def _context_steps(wl, seed, dt, stream):
    p = wl.pulses[0]
    cfg, keep = chem.make_config(wl.L, wl.D, wl.reactions, seed=seed, precision=chem.CHEM_FP64,
                                 dt_min=dt, dt_max=dt, capacity_species=8192,
                                 capacity_event_log=1 << 14, stream=stream)
    ctx = chem.chem_init(cfg)
    out = []
    try:
        chem.chem_inject_pulse(ctx, p.types, p.xyz, p.t_arrival, p.energy_eV)
        for k in (1, 2):
            chem.chem_run_until(ctx, k * dt)
            ids, types, xyz = chem.chem_get_state(ctx)
            o = np.argsort(ids)
            ev = chem.chem_get_events(ctx)
            # ids handed out so far: the released species (all at t = 0), then every product
            next_id = p.n + int(ev["n_prod"].sum())
            out.append((ids[o].astype(np.int64), types[o].astype(np.int64), xyz[o],
                        event_matrix(ev[ev["step"] == k - 1]), next_id))
    finally:
        chem.chem_destroy(ctx)
    return out


def test_two_noalloc_steps_match_the_context_path():
    import torch
    seed, dt = 8, 1e-9
    wl = W.uniform_2000(seed=seed, L=200.0, n_steps=2)
    p = wl.pulses[0]
    n = p.n
    stream = torch.cuda.current_stream().cuda_stream
    ref = _context_steps(wl, seed, dt, stream)

    M = chem.CHEM_NOALLOC_MAX_SPECIES
    dev = torch.device("cuda", 0)
    cfg, keep = chem.make_config(wl.L, wl.D, wl.reactions, seed=seed, precision=chem.CHEM_FP64,
                                 dt_min=dt, dt_max=dt, stream=stream)
    ids = torch.arange(n, dtype=torch.int32, device=dev)
    types = torch.from_numpy(p.types.astype(np.int32)).to(dev)
    xyz = torch.from_numpy(np.ascontiguousarray(p.xyz)).to(dev)
    next_id = n
    ev_words = ctypes.sizeof(chem.chem_event) // 4
    for k in range(2):
        id_out = torch.empty(M, dtype=torch.int32, device=dev)
        type_out = torch.empty(M, dtype=torch.int32, device=dev)
        xyz_out = torch.empty((M, 3), dtype=torch.float64, device=dev)
        n_out = torch.zeros(1, dtype=torch.int32, device=dev)
        next_out = torch.zeros(1, dtype=torch.int32, device=dev)
        ev_out = torch.empty((M // 2) * ev_words, dtype=torch.int32, device=dev)
        n_ev = torch.zeros(1, dtype=torch.int32, device=dev)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info(0)[0]
        torch_before = torch.cuda.memory_allocated(0)
        st = chem.chem_step_noalloc(cfg, k, k * dt, dt, next_id, ids.numel(), ids.data_ptr(),
                                    types.data_ptr(), xyz.data_ptr(), id_out.data_ptr(),
                                    type_out.data_ptr(), xyz_out.data_ptr(), n_out.data_ptr(),
                                    next_out.data_ptr(), ev_out.data_ptr(), n_ev.data_ptr())
        assert st == chem.CHEM_OK, chem.STATUS_NAMES.get(st, st)
        if k == 1:
            # the second call (its kernels already loaded by the first) allocates nothing:
            # neither the device's free memory nor torch's pool moves
            assert torch.cuda.mem_get_info(0)[0] == free_before
            assert torch.cuda.memory_allocated(0) == torch_before
        m = int(n_out.item())
        got_ids = id_out[:m].cpu().numpy().astype(np.int64)
        got_types = type_out[:m].cpu().numpy().astype(np.int64)
        got_xyz = xyz_out[:m].cpu().numpy()
        o = np.argsort(got_ids)
        r_ids, r_types, r_xyz, r_ev, r_next = ref[k]
        assert np.array_equal(got_ids[o], r_ids)
        assert np.array_equal(got_types[o], r_types)
        d = got_xyz[o] - r_xyz
        d -= wl.L * np.round(d / wl.L)
        assert np.abs(d).max() <= 1e-12 * wl.L
        ne = int(n_ev.item())
        ev = ev_out[:ne * ev_words].cpu().numpy().view(chem.EVENT_DTYPE)
        assert np.array_equal(event_matrix(ev), r_ev)
        assert ne > 0
        assert int(next_out.item()) == r_next
        # feed this step's output to the next call
        ids, types, xyz = id_out[:m].clone(), type_out[:m].clone(), xyz_out[:m].clone()
        next_id = int(next_out.item())


def test_noalloc_rejects_sizes_beyond_its_fixed_array():
    import torch
    wl = W.uniform_2000(seed=1, L=200.0)
    cfg, keep = chem.make_config(wl.L, wl.D, wl.reactions, seed=1, precision=chem.CHEM_FP64,
                                 dt_min=1e-9, dt_max=1e-9,
                                 stream=torch.cuda.current_stream().cuda_stream)
    dummy = torch.zeros(16, dtype=torch.int64, device="cuda")
    a = dummy.data_ptr()
    st = chem.chem_step_noalloc(cfg, 0, 0.0, 1e-9, 0, chem.CHEM_NOALLOC_MAX_SPECIES + 1,
                                a, a, a, a, a, a, a, a, a, a)
    assert st == chem.CHEM_ECAPACITY


def test_noalloc_rejects_bad_device_inputs():
    # The species live on the device, so the entry point checks them there: a type equal
    # to n_types (7 for the water table) returns CHEM_EINVAL and writes no species.
    import torch
    wl = W.uniform_2000(seed=2, L=200.0)
    p = wl.pulses[0]
    stream = torch.cuda.current_stream().cuda_stream
    cfg, keep = chem.make_config(wl.L, wl.D, wl.reactions, seed=2, precision=chem.CHEM_FP64,
                                 dt_min=1e-9, dt_max=1e-9, stream=stream)
    dev = torch.device("cuda", 0)
    n = p.n
    M = chem.CHEM_NOALLOC_MAX_SPECIES
    ev_words = ctypes.sizeof(chem.chem_event) // 4
    ids = torch.arange(n, dtype=torch.int32, device=dev)
    good_types = torch.from_numpy(p.types.astype(np.int32)).to(dev)
    xyz = torch.from_numpy(np.ascontiguousarray(p.xyz)).to(dev)
    bad_types = good_types.clone()
    bad_types[n // 2] = 7
    bad_xyz = xyz.clone()
    bad_xyz[3, 1] = float("nan")
    for types, pos in ((bad_types, xyz), (good_types, bad_xyz)):
        id_out = torch.empty(M, dtype=torch.int32, device=dev)
        type_out = torch.empty(M, dtype=torch.int32, device=dev)
        xyz_out = torch.empty((M, 3), dtype=torch.float64, device=dev)
        n_out = torch.full((1,), -1, dtype=torch.int32, device=dev)
        next_out = torch.zeros(1, dtype=torch.int32, device=dev)
        ev_out = torch.empty((M // 2) * ev_words, dtype=torch.int32, device=dev)
        n_ev = torch.full((1,), -1, dtype=torch.int32, device=dev)
        st = chem.chem_step_noalloc(cfg, 0, 0.0, 1e-9, n, n, ids.data_ptr(), types.data_ptr(),
                                    pos.data_ptr(), id_out.data_ptr(), type_out.data_ptr(),
                                    xyz_out.data_ptr(), n_out.data_ptr(), next_out.data_ptr(),
                                    ev_out.data_ptr(), n_ev.data_ptr())
        assert st == chem.CHEM_EINVAL
        assert int(n_out.item()) == 0 and int(n_ev.item()) == 0 and int(next_out.item()) == n
    # a good call right after still works (the status does not stick to the array)
    id_out = torch.empty(M, dtype=torch.int32, device=dev)
    type_out = torch.empty(M, dtype=torch.int32, device=dev)
    xyz_out = torch.empty((M, 3), dtype=torch.float64, device=dev)
    n_out = torch.zeros(1, dtype=torch.int32, device=dev)
    next_out = torch.zeros(1, dtype=torch.int32, device=dev)
    ev_out = torch.empty((M // 2) * ev_words, dtype=torch.int32, device=dev)
    n_ev = torch.zeros(1, dtype=torch.int32, device=dev)
    st = chem.chem_step_noalloc(cfg, 0, 0.0, 1e-9, n, n, ids.data_ptr(), good_types.data_ptr(),
                                xyz.data_ptr(), id_out.data_ptr(), type_out.data_ptr(),
                                xyz_out.data_ptr(), n_out.data_ptr(), next_out.data_ptr(),
                                ev_out.data_ptr(), n_ev.data_ptr())
    assert st == chem.CHEM_OK and int(n_out.item()) > 0
