"""fgi_integrate_h_static: H integration for callers that cannot allocate.

Some callers cannot call cudaMalloc or pass a workspace (a Fortran SCF driver
without a CUDA allocator, a plug-in inside another framework's memory pool,
code that must not allocate inside its loop).  The static entry point keeps
its scratch in a fixed-size device array inside the library.  These checks
call it through the C ABI and compare it with fgi_integrate_h (caller
workspace), twice in a row, and check that a plan larger than the array is
refused with a clear error.
"""
import ctypes as C

import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fgi():
    from paper_2208_12335_gb300 import build as B
    B.build()
    import paper_2208_12335_gb300 as P
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return P


def _call_static(fgi, ctx, v, h, accumulate=0):
    lib = fgi.lib()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.fgi_integrate_h_static(ctx._h, C.c_void_p(v.data_ptr()), C.c_void_p(h.data_ptr()),
                                      accumulate, stream)


@pytest.mark.parametrize("precision,tol", [("split_bf16", 1e-12), ("fp64", 1e-11)])
def test_static_scratch_matches_workspace_entry_point(fgi, precision, tol):
    prob = W.tiny_water()
    ctx = fgi.Context(0).load(prob, precision)
    v = torch.from_numpy(prob.v).cuda()
    ref = ctx.integrate_h(v).clone()
    ctx.sync()
    scale = ref.abs().max().item()
    for _ in range(2):                                     # two calls in a row
        h = torch.full_like(ref, float("nan"))
        assert _call_static(fgi, ctx, v, h) == 0, fgi.lib().fgi_last_error(ctx._h)
        ctx.sync()
        assert (h - ref).abs().max().item() <= tol * scale
    # accumulate = 1 adds onto what is there
    h2 = ref.clone()
    assert _call_static(fgi, ctx, v, h2, 1) == 0
    ctx.sync()
    assert (h2 - 2 * ref).abs().max().item() <= 2 * tol * scale


def test_static_scratch_refuses_plans_beyond_its_size(fgi):
    prob = W.tiny_water(n_rad=80, n_ang=302)
    ctx = fgi.Context(0).load(prob, "split_bf16")
    assert ctx.workspace_size() > fgi.fgi.FGI_STATIC_SCRATCH_BYTES
    v = torch.from_numpy(prob.v).cuda()
    h = torch.empty(ctx.sizes()[1], dtype=torch.float64, device="cuda")
    rc = _call_static(fgi, ctx, v, h)
    assert rc == -4
    assert b"static scratch holds" in fgi.lib().fgi_last_error(ctx._h)
