"""Device-side failure reporting (GPU).

Every kernel bounds its waits; a wait that runs out makes the kernel wind
down and write an error code into a host-mapped error word, which the host
entry points turn into PFB_ERR_TIMEOUT.  The failure is made with the test
hook pfb_plan_set_fault: the producer role of the single-CTA warp-specialised
FFT kernel issues no input copies, so its consumers' waits (bounded here at
2 ms) run out.  Nothing faults or hangs the GPU: no memory is touched, no
copy is in flight, and every role leaves its loop after its bounded wait.
The same plan must then run normally again and match the FP64 oracle.
"""

import numpy as np
import pytest

import paper_2408_16551_gb300 as pkg
from paper_2408_16551_gb300 import synth

from gpu_common import TOL_F32, TOL_MAX_F32, assert_close, reference, to_device

pytestmark = pytest.mark.gpu

WAIT_NS = 2_000_000  # 2 ms


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_16551_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _plan():
    plan = pkg.Plan(1024, 16, pkg.PFB_IN_C64, pkg.PFB_WIN_HAMMING)
    plan.variant = 5  # the single-CTA warp-specialised kernel, which honours the hook
    return plan


def test_timeout_reported_by_host_calls_then_plan_recovers():
    P, T = 1024, 16
    plan = _plan()
    x = synth.small_stream(P, T, P * (T - 1 + 300) + 3, seed=51).generate()
    ref = reference(x, synth.IN_C64, P, T, synth.WIN_HAMMING)
    plan.set_fault(1, WAIT_NS)
    for call in (plan.execute_host, plan.execute_host_noalloc):
        with pytest.raises(pkg.PFBError) as e:
            call(x)
        assert e.value.status == pkg.PFB_ERR_TIMEOUT, call.__name__
        assert plan.status() == pkg.PFB_OK  # the call read and cleared the word
    plan.set_fault(0)
    for call in (plan.execute_host, plan.execute_host_noalloc):
        assert_close(call(x), ref, TOL_F32, TOL_MAX_F32, what=call.__name__)
    assert plan.status() == pkg.PFB_OK
    plan.close()


def test_timeout_reported_by_plan_status_after_async_execute():
    import torch
    P, T = 1024, 16
    plan = _plan()
    x = synth.small_stream(P, T, P * (T - 1 + 200) + 7, seed=52).generate()
    xd = to_device(x)
    plan.set_fault(1, WAIT_NS)
    plan.execute(xd)
    torch.cuda.synchronize()
    assert plan.status() == pkg.PFB_ERR_TIMEOUT
    assert plan.status() == pkg.PFB_OK  # read and cleared
    plan.set_fault(0)
    X = plan.execute(xd)
    torch.cuda.synchronize()
    assert plan.status() == pkg.PFB_OK
    assert_close(X.cpu().numpy(), reference(x, synth.IN_C64, P, T, synth.WIN_HAMMING), TOL_F32, TOL_MAX_F32)
    plan.close()


def test_timeout_fails_the_server_request_and_the_stream_continues():
    """A served chunk whose kernel timed out reports PFB_ERR_TIMEOUT through
    pfb_wait/pfb_poll (the batch's own error word); the stream's resident
    state is still advanced, so the next chunk's spectra equal the oracle's."""
    import torch
    P, T = 1024, 16
    plan = _plan()
    n1, n2 = P * 64, P * 48
    x = synth.small_stream(P, T, n1 + n2, seed=53).generate()
    ref = reference(x, synth.IN_C64, P, T, synth.WIN_HAMMING)
    srv = pkg.Server(hbm_budget_bytes=1 << 30, max_slots=4, timeout_ms=5000)
    sid = srv.open_stream(plan)
    xd = to_device(x)
    S1, S2 = srv.next_spectra(sid, n1), None
    o1 = torch.empty((S1, P), dtype=torch.complex64, device="cuda")
    plan.set_fault(1, WAIT_NS)
    t1 = srv.submit(sid, xd[:n1], n1, o1)
    assert srv.wait(t1, 10000) == pkg.PFB_ERR_TIMEOUT
    assert srv.poll(t1) == pkg.PFB_ERR_TIMEOUT
    plan.set_fault(0)
    S2 = srv.next_spectra(sid, n2)
    o2 = torch.empty((S2, P), dtype=torch.complex64, device="cuda")
    t2 = srv.submit(sid, xd[n1:], n2, o2)
    assert srv.wait(t2, 10000) == pkg.PFB_OK
    assert_close(o2.cpu().numpy(), ref[S1:S1 + S2], TOL_F32, TOL_MAX_F32, what="chunk after the failed one")
    st = srv.stats()
    assert st["failed"] == 1 and st["completed"] == 1
    srv.close_stream(sid)
    srv.close()
    plan.close()


def test_set_fault_rejects_bad_arguments():
    plan = _plan()
    for mode, ns in ((2, 0), (-1, 0), (1, -5), (0, 5_000_000_000)):
        with pytest.raises(pkg.PFBError) as e:
            plan.set_fault(mode, ns)
        assert e.value.status == pkg.PFB_ERR_INVALID
    plan.close()
