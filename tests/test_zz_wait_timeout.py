"""Failure detection on the GPU without a fault.

Every wait of the pipelined kernels on an mbarrier is bounded in time; when
one runs out the kernel records a time-out in the context's status word and
returns instead of hanging.  fgi_selftest_wait_timeout launches one small
kernel whose wait on a barrier that nothing completes must run out that way:
the next sync raises FGI_ERR_TIMEOUT after the bounded time, clears the
status, and the context then computes the same H as before.
"""
import time

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


def test_bounded_wait_runs_out_and_the_context_stays_usable(fgi):
    prob = W.tiny_water(n_rad=16, n_ang=26)
    ctx = fgi.Context(0).load(prob, "split_bf16")
    v = torch.from_numpy(prob.v).to("cuda:0")
    h0 = ctx.integrate_h(v).clone()
    ctx.sync()
    t0 = time.perf_counter()
    ctx.selftest_wait_timeout()
    with pytest.raises(fgi.FGIError) as e:
        ctx.sync()
    waited = time.perf_counter() - t0
    assert e.value.code == -5                        # FGI_ERR_TIMEOUT
    assert 1.0 < waited < 60.0                       # the 2 s device limit, not a hang
    ctx.sync()                                       # the status word was cleared
    h1 = ctx.integrate_h(v).clone()
    ctx.sync()
    assert torch.equal(h0, h1)                       # fixed-point sums: bitwise the same
