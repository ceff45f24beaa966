"""The allocation-free totals entry point (for callers that cannot let the library allocate device
memory), called through the C ABI and checked against the allocating vga_sim_totals on two calls in
a row.  This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

HEADER_BYTES = 32  # vga_sim_save_state: header, then 5n FP32 values, then 5n BF16 residuals


def test_noalloc_totals_match_allocating_entry_point(vga):
    import torch

    img = synth.pore_mask((40, 36, 44), 0.22, 21)
    g = vga.Graph(img)
    kept = synth.kept_mask_from_nodes(img.shape, g.export(labels=False, nbr=False)["voxel_of_node"])
    X0 = synth.initial_masses(kept, 21, with_organic_matter=True)
    sim = vga.Sim(g, synth.paper_params())
    sim.set_masses(X0)
    n = g.n
    lib = vga.load_library()
    stream = torch.cuda.current_stream()
    totals = torch.full((5,), np.nan, dtype=torch.float64, device="cuda")
    for _ in range(2):
        sim.step(50)
        ref = sim.totals()
        raw = sim.save_state()
        vals = np.frombuffer(raw, dtype=np.float32, count=5 * n, offset=HEADER_BYTES)
        res = np.frombuffer(raw, dtype=np.uint16, count=5 * n, offset=HEADER_BYTES + 20 * n)
        d_vals = torch.from_numpy(vals.copy()).cuda()
        d_res = torch.from_numpy(res.view(np.int16).copy()).cuda()
        torch.cuda.synchronize()
        status = lib.vga_state_totals_noalloc(C.c_void_p(d_vals.data_ptr()), C.c_void_p(d_res.data_ptr()), n, n,
                                              C.c_void_p(totals.data_ptr()), C.c_void_p(stream.cuda_stream))
        assert status == 0, vga.vga_last_error()
        torch.cuda.synchronize()
        got = totals.cpu().numpy()
        assert np.allclose(got, ref, rtol=1e-12, atol=0), (got, ref)
        # values alone (no residuals) differ from the full pair only at the FP32 rounding level
        vga.vga_state_totals_noalloc(d_vals, None, n, n, totals, stream)
        torch.cuda.synchronize()
        assert np.allclose(totals.cpu().numpy(), ref, rtol=1e-6, atol=0)


def test_noalloc_rejects_sizes_beyond_its_scratch(vga):
    lib = vga.load_library()
    dummy = C.c_void_p(16)  # never dereferenced: the size checks come first
    limit = 4096 * 8192
    assert lib.vga_state_totals_noalloc(dummy, None, limit + 1, limit + 1, dummy, None) == -1
    assert "no-allocation limit" in vga.vga_last_error()
    assert lib.vga_state_totals_noalloc(dummy, None, 10, 9, dummy, None) == -1
    assert lib.vga_state_totals_noalloc(None, None, 10, 10, dummy, None) == -1


def _host_totals(vals, res, n, stride):
    """Exact sums (math.fsum) of value + decoded BF16 residual per compartment."""
    import math

    out = []
    for c in range(5):
        v = vals[c * stride: c * stride + n].astype(np.float64)
        if res is not None:
            r = (res[c * stride: c * stride + n].astype(np.uint32) << 16).view(np.float32).astype(np.float64)
            v = np.concatenate([v, r])
        out.append(math.fsum(v.tolist()))
    return np.array(out)


def test_noalloc_strided_empty_and_block_boundary(vga):
    """Row strides above n with the padding filled with NaN (it must never be read), n = 0 (only the
    final reduction runs: exact zeros), and n = 2 * 8192 + 1 (one node past a block boundary), each
    twice in a row, against exact host sums of the same values."""
    import torch

    img = synth.pore_mask((48, 48, 48), 0.26, 5)
    g = vga.Graph(img)
    kept = synth.kept_mask_from_nodes(img.shape, g.export(labels=False, nbr=False)["voxel_of_node"])
    sim = vga.Sim(g, synth.paper_params())
    sim.set_masses(synth.initial_masses(kept, 5, with_organic_matter=True))
    sim.step(20)
    N = g.n
    assert N > 2 * 8192 + 1
    raw = sim.save_state()
    vals = np.frombuffer(raw, dtype=np.float32, count=5 * N, offset=HEADER_BYTES).reshape(5, N)
    res = np.frombuffer(raw, dtype=np.uint16, count=5 * N, offset=HEADER_BYTES + 20 * N).reshape(5, N)
    stream = torch.cuda.current_stream()
    totals = torch.empty((5,), dtype=torch.float64, device="cuda")
    # (n = 0 still passes real buffers: the entry point rejects NULL pointers whatever n is)
    for n, pad in ((N, 37), (2 * 8192 + 1, 0), (2 * 8192 + 1, 91), (0, 1), (0, 5)):
        stride = n + pad
        hv = np.full((5, stride), np.nan, dtype=np.float32)
        hr = np.full((5, stride), 0x7fc0, dtype=np.uint16)  # BF16 NaN in the padding
        hv[:, :n] = vals[:, :n]
        hr[:, :n] = res[:, :n]
        hv, hr = hv.ravel(), hr.ravel()
        want = _host_totals(hv, hr, n, stride)
        d_vals = torch.from_numpy(hv.copy()).cuda()
        d_res = torch.from_numpy(hr.view(np.int16).copy()).cuda()
        for _ in range(2):
            totals.fill_(np.nan)
            vga.vga_state_totals_noalloc(d_vals, d_res, n, stride, totals, stream)
            torch.cuda.synchronize()
            got = totals.cpu().numpy()
            if n == 0:
                assert got.tolist() == [0.0] * 5
            else:
                assert np.allclose(got, want, rtol=1e-12, atol=0), (n, stride, got, want)
