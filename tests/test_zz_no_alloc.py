"""The allocation-free operator entry point (hh_apply_operator_noalloc).

It serves callers that cannot allocate device memory (code inside a memory
pool or arena it does not own, allocation-free real-time loops, hosts whose
allocator must not be re-entered): the caller passes device inputs and
outputs, and the library's scratch is a fixed device array. This test calls
it through the C ABI twice in a row and compares each result with the
allocating hh_apply_operator, within the FP32 operator tolerance the other
parity tests use. The file is named so that pytest collects it last.
"""

import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

PH = synth.PHASES_SOLID_CLAY_PORE


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def test_noalloc_operator_matches_allocating_entry_point():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("a GPU test ran without a CUDA device")
    from paper_2208_02320_gb300 import Context, _build, binding
    _build.build()
    lib = binding.load()
    rng = np.random.default_rng(2208)
    phases, nph = binding._phases(PH)
    stream = torch.cuda.current_stream()
    with Context(0) as ctx:
        for call, shape in enumerate([(12, 18, 20), (24, 26, 22)]):
            lab = rng.integers(0, len(PH), size=shape).astype(np.uint8)
            p = rng.standard_normal((6,) + shape)
            ref = ctx.apply_operator(p, labels=lab, phases=PH, precision="fp32")
            d_lab = torch.from_numpy(lab).cuda()
            d_p = torch.from_numpy(p.astype(np.float32)).cuda()
            d_q = torch.full_like(d_p, float("nan"))
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            nz, ny, nx = shape
            s = lib.hh_apply_operator_noalloc(ctypes.c_void_p(d_lab.data_ptr()), phases, nph, nx, ny, nz,
                                              ctypes.c_void_p(d_p.data_ptr()), ctypes.c_void_p(d_q.data_ptr()),
                                              binding.HH_NYQ_ZERO_COMPONENT, ctypes.c_void_p(stream.cuda_stream))
            assert s == binding.HH_OK, lib.hh_last_error(None)
            free1 = torch.cuda.mem_get_info()[0]
            if call > 0:
                # the device address lookup happened on the first call; later
                # calls leave free device memory exactly unchanged
                assert free1 == free0
            q = d_q.cpu().numpy().astype(np.float64)
            assert np.isfinite(q).all()
            assert _rel(q, ref) < 2e-5, call


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("a GPU test ran without a CUDA device")
    from paper_2208_02320_gb300 import binding
    lib = binding.load()
    phases, nph = binding._phases(PH)
    d = torch.zeros(8, dtype=torch.float32, device="cuda")
    lab = torch.zeros(8, dtype=torch.uint8, device="cuda")
    big = 96  # above the per-edge limit
    s = lib.hh_apply_operator_noalloc(ctypes.c_void_p(lab.data_ptr()), phases, nph, big, 8, 8,
                                      ctypes.c_void_p(d.data_ptr()), ctypes.c_void_p(d.data_ptr()),
                                      binding.HH_NYQ_ZERO_COMPONENT, None)
    assert s == binding.HH_ERR_ARG
    assert b"HH_NOALLOC_MAX_EDGE" in lib.hh_last_error(None)


def test_noalloc_rejects_a_label_outside_the_phase_table():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("a GPU test ran without a CUDA device")
    from paper_2208_02320_gb300 import binding
    lib = binding.load()
    phases, nph = binding._phases(PH)
    shape = (8, 8, 8)
    lab = torch.zeros(shape, dtype=torch.uint8, device="cuda")
    lab[3, 4, 5] = nph  # one past the table
    p = torch.zeros((6,) + shape, dtype=torch.float32, device="cuda")
    q = torch.zeros_like(p)
    stream = torch.cuda.current_stream()
    s = lib.hh_apply_operator_noalloc(ctypes.c_void_p(lab.data_ptr()), phases, nph, 8, 8, 8,
                                      ctypes.c_void_p(p.data_ptr()), ctypes.c_void_p(q.data_ptr()),
                                      binding.HH_NYQ_ZERO_COMPONENT, ctypes.c_void_p(stream.cuda_stream))
    assert s == binding.HH_ERR_ARG
    assert b"label" in lib.hh_last_error(None)
    # the flag does not stick: a valid call right after succeeds
    lab[3, 4, 5] = nph - 1
    s = lib.hh_apply_operator_noalloc(ctypes.c_void_p(lab.data_ptr()), phases, nph, 8, 8, 8,
                                      ctypes.c_void_p(p.data_ptr()), ctypes.c_void_p(q.data_ptr()),
                                      binding.HH_NYQ_ZERO_COMPONENT, ctypes.c_void_p(stream.cuda_stream))
    assert s == binding.HH_OK, lib.hh_last_error(None)
