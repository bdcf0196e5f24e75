"""Serving: resident filter state, continuous batching, admission, faults
injected on the host (no GPU fault is provoked)."""

import os
import time

import numpy as np
import pytest

import paper_2408_16551_gb300 as pkg
from paper_2408_16551_gb300 import synth

from gpu_common import assert_close, reference, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_16551_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _chunked(server, plan, x, chunk):
    """Submit x in chunks of `chunk` samples; return the concatenated outputs."""
    import torch
    sid = server.open_stream(plan)
    per = 2 if plan.in_dtype == pkg.PFB_IN_CI8 else 1
    n = x.numel() // per
    outs, tickets = [], []
    for c0 in range(0, n, chunk):
        part = x[c0 * per:(c0 + chunk) * per]
        S = server.next_spectra(sid, chunk)
        out = torch.empty((max(S, 1), plan.P), dtype=torch.complex64, device="cuda")
        tickets.append(server.submit(sid, part, chunk, out))
        outs.append(out[:S])
    for t in tickets:
        assert server.wait(t, 20000) == pkg.PFB_OK
    server.close_stream(sid)
    return torch.cat(outs)


@pytest.mark.parametrize("P,T,dt,chunk,nchunks", [(1024, 16, synth.IN_C64, 1 << 14, 9),
                                                  (4096, 16, synth.IN_CI8, 1 << 16, 4),
                                                  (256, 8, synth.IN_C64, 256 * 3, 11),
                                                  (64, 16, synth.IN_R32, 64 * 5, 12)])
def test_chunked_stream_equals_whole_stream(P, T, dt, chunk, nchunks):
    import torch
    n = chunk * nchunks
    x = synth.small_stream(P, T, n, in_dtype=dt, seed=P).generate()
    xd = to_device(x)
    plan = pkg.Plan(P, T, dt, pkg.PFB_WIN_BLACKMAN)
    whole = plan.execute(xd)
    srv = pkg.Server(hbm_budget_bytes=1 << 32, max_slots=4)
    got = _chunked(srv, plan, xd, chunk)
    torch.cuda.synchronize()
    assert got.shape == whole.shape
    assert torch.equal(got, whole)          # same kernel, same summation order
    assert_close(got.cpu().numpy(), reference(x, dt, P, T, synth.WIN_BLACKMAN), what="chunked vs oracle")
    assert srv.close() == pkg.PFB_OK


def test_alone_equals_in_mix():
    import torch
    P, T, chunk = 1024, 16, 1 << 14
    plan = pkg.Plan(P, T)
    xs = [to_device(synth.small_stream(P, T, chunk * 6, seed=40 + i).generate()) for i in range(6)]
    srv = pkg.Server(hbm_budget_bytes=1 << 32, max_slots=8)
    alone = _chunked(srv, plan, xs[0], chunk)
    # now stream 0 again, interleaved with five other streams in flight
    sids = [srv.open_stream(plan) for _ in xs]
    outs = [[] for _ in xs]
    tickets = []
    for c in range(6):
        for i, sid in enumerate(sids):
            S = srv.next_spectra(sid, chunk)
            out = torch.empty((S, P), dtype=torch.complex64, device="cuda")
            tickets.append(srv.submit(sid, xs[i][c * chunk:(c + 1) * chunk], chunk, out))
            outs[i].append(out)
    for t in tickets:
        assert srv.wait(t, 20000) == pkg.PFB_OK
    mixed = torch.cat(outs[0])
    assert torch.equal(mixed, alone)
    st = srv.stats()
    assert st["completed"] == 6 + 36 and st["failed"] == 0
    assert st["p99_latency_us"] >= st["p50_latency_us"] > 0
    assert srv.close() == pkg.PFB_OK


def test_admission_by_budget_queues_and_completes():
    import torch
    P, T, chunk = 1024, 16, 1 << 14
    plan = pkg.Plan(P, T)
    req_bytes = chunk * 8 + (chunk // P) * P * 8
    state_bytes = 2 * (T - 1) * P * 8
    nstreams = 4
    budget = nstreams * state_bytes + 2 * req_bytes       # at most two requests on the device
    srv = pkg.Server(hbm_budget_bytes=budget, max_slots=8, queue_when_busy=True)
    sids = [srv.open_stream(plan) for _ in range(nstreams)]
    x = to_device(synth.small_stream(P, T, chunk, seed=1).generate())
    tickets = []
    for rep in range(5):
        for sid in sids:
            S = srv.next_spectra(sid, chunk)
            out = torch.empty((max(S, 1), P), dtype=torch.complex64, device="cuda")
            tickets.append((srv.submit(sid, x, chunk, out), out))
    for t, _ in tickets:
        assert srv.wait(t, 20000) == pkg.PFB_OK
    st = srv.stats()
    assert st["peak_reserved_bytes"] <= budget
    assert st["completed"] == 20
    assert srv.close() == pkg.PFB_OK


def test_busy_when_not_queuing():
    import torch
    P, T, chunk = 4096, 16, 1 << 16
    plan = pkg.Plan(P, T)
    srv = pkg.Server(hbm_budget_bytes=1 << 32, max_slots=1, queue_when_busy=False)
    sid = srv.open_stream(plan)
    big = to_device(synth.small_stream(P, T, chunk * 64, seed=2).generate())
    got_busy = False
    tickets = []
    for c in range(64):
        S = srv.next_spectra(sid, chunk)
        out = torch.empty((max(S, 1), P), dtype=torch.complex64, device="cuda")
        try:
            tickets.append(srv.submit(sid, big[c * chunk:(c + 1) * chunk], chunk, out))
        except pkg.PFBError as e:
            assert e.status == pkg.PFB_ERR_BUSY
            got_busy = True
            break
    for t in tickets:
        assert srv.wait(t, 20000) == pkg.PFB_OK
    assert got_busy
    assert srv.stats()["rejected"] >= 1
    srv.close()


def test_invalid_submissions():
    import torch
    plan = pkg.Plan(1024, 16)
    srv = pkg.Server(hbm_budget_bytes=1 << 30, max_slots=2)
    sid = srv.open_stream(plan)
    x = torch.zeros(1024 * 20 + 5, dtype=torch.complex64, device="cuda")
    out = torch.empty((20, 1024), dtype=torch.complex64, device="cuda")
    with pytest.raises(pkg.PFBError) as ei:
        srv.submit(sid, x, 1024 * 20 + 5, out)            # not a multiple of P
    assert ei.value.status == pkg.PFB_ERR_INVALID
    with pytest.raises(pkg.PFBError):
        srv.submit(sid + 100, x, 1024 * 20, out)            # unknown stream
    with pytest.raises(pkg.PFBError):
        srv.submit(sid, x, 1024 * 20, out[:1])              # output too small
    srv.close()


def test_injected_launch_failure_fails_only_that_request(monkeypatch):
    import torch
    monkeypatch.setenv("PFB_FAULT", "launch_fail:3")
    P, T, chunk = 1024, 16, 1 << 13
    plan = pkg.Plan(P, T)
    srv = pkg.Server(hbm_budget_bytes=1 << 32, max_slots=4)
    monkeypatch.delenv("PFB_FAULT")
    sids = [srv.open_stream(plan) for _ in range(5)]
    x = to_device(synth.small_stream(P, T, chunk, seed=3).generate())
    tickets = []
    for sid in sids:
        out = torch.empty((max(srv.next_spectra(sid, chunk), 1), P), dtype=torch.complex64, device="cuda")
        tickets.append((srv.submit(sid, x, chunk, out), out))
    res = [srv.wait(t, 20000) for t, _ in tickets]
    assert res.count(pkg.PFB_ERR_CUDA) == 1 and res.count(pkg.PFB_OK) == 4
    assert res[2] == pkg.PFB_ERR_CUDA
    st = srv.stats()
    assert st["failed"] == 1 and st["completed"] == 4
    assert srv.close() == pkg.PFB_OK


def test_lost_completion_times_out(monkeypatch):
    import torch
    monkeypatch.setenv("PFB_FAULT", "lose_completion:2")
    P, T, chunk = 256, 8, 256 * 16
    plan = pkg.Plan(P, T)
    srv = pkg.Server(hbm_budget_bytes=1 << 30, max_slots=4, timeout_ms=200)
    monkeypatch.delenv("PFB_FAULT")
    sids = [srv.open_stream(plan) for _ in range(3)]
    x = to_device(synth.small_stream(P, T, chunk, seed=4).generate())
    tickets = []
    for sid in sids:
        out = torch.empty((max(srv.next_spectra(sid, chunk), 1), P), dtype=torch.complex64, device="cuda")
        tickets.append((srv.submit(sid, x, chunk, out), out))
    res = [srv.wait(t, 5000) for t, _ in tickets]
    assert res == [pkg.PFB_OK, pkg.PFB_ERR_TIMEOUT, pkg.PFB_OK]
    # the lost request still holds its slot, so destroy reports a timeout
    assert srv.close() == pkg.PFB_ERR_TIMEOUT


@pytest.mark.parametrize("P,T,dt,chunk,split", [(1024, 16, synth.IN_C64, 1 << 13, 3),   # state = T-1 frames
                                                (4096, 16, synth.IN_CI8, 4096 * 4, 2),  # 8 frames < T-1
                                                (256, 8, synth.IN_R32, 256 * 5, 0),     # exported before any chunk
                                                (64, 4, synth.IN_C64, 64 * 2, 1)])
def test_state_export_import_resumes_bitwise(P, T, dt, chunk, split):
    """Checkpoint: a stream's filter state exported after `split` chunks and
    imported into a fresh stream (on a fresh server) continues it exactly: the
    spectra of both halves equal the uninterrupted stream bit for bit."""
    import torch
    nchunks = 7
    per = 2 if dt == synth.IN_CI8 else 1
    x = to_device(synth.small_stream(P, T, chunk * nchunks, in_dtype=dt, seed=P + split).generate())
    plan = pkg.Plan(P, T, dt, pkg.PFB_WIN_HAMMING)
    whole = plan.execute(x)
    outs = []

    def run(srv, sid, c_from, c_to):
        tickets = []
        for c in range(c_from, c_to):
            S = srv.next_spectra(sid, chunk)
            out = torch.empty((max(S, 1), P), dtype=torch.complex64, device="cuda")
            tickets.append(srv.submit(sid, x[c * chunk * per:(c + 1) * chunk * per], chunk, out))
            outs.append(out[:S])
        for t in tickets:
            assert srv.wait(t, 20000) == pkg.PFB_OK

    a = pkg.Server(hbm_budget_bytes=1 << 32, max_slots=4)
    sa = a.open_stream(plan)
    run(a, sa, 0, split)
    blob = a.export_state(sa)
    assert len(blob) == 48 + min(T - 1, split * chunk // P) * P * (8 if dt == synth.IN_C64 else (2 if dt == synth.IN_CI8 else 4))
    a.close_stream(sa)
    a.close()
    b = pkg.Server(hbm_budget_bytes=1 << 32, max_slots=4)
    sb = b.open_stream(plan)
    b.import_state(sb, blob)
    run(b, sb, split, nchunks)
    torch.cuda.synchronize()
    got = torch.cat(outs)
    assert got.shape == whole.shape
    assert torch.equal(got, whole)
    b.close_stream(sb)
    b.close()


def test_state_import_rejects_foreign_blobs():
    P, T = 1024, 16
    srv = pkg.Server(hbm_budget_bytes=1 << 32, max_slots=4)
    p1 = pkg.Plan(P, T, pkg.PFB_IN_C64)
    p2 = pkg.Plan(P, 8, pkg.PFB_IN_C64)
    s1, s2 = srv.open_stream(p1), srv.open_stream(p2)
    blob = srv.export_state(s1)
    with pytest.raises(pkg.PFBError) as e:
        srv.import_state(s2, blob)                     # another T
    assert e.value.status == pkg.PFB_ERR_INVALID
    with pytest.raises(pkg.PFBError):
        srv.import_state(s1, b"x" * len(blob))         # not a state blob
    with pytest.raises(pkg.PFBError):
        srv.import_state(s1, blob[:20])                # shorter than its header
    srv.import_state(s1, blob)                         # its own blob is fine
    srv.close_stream(s1)
    srv.close_stream(s2)
    srv.close()


def test_submit_chunks_equals_single_submits_and_ticket_times():
    """pfb_submit_chunks (n chunks of one buffer in one call) gives the same
    spectra as chunk-by-chunk submission, bit for bit; pfb_ticket_times
    reports the server's submit and completion times on the steady clock."""
    import torch
    P, T, chunk, nch = 4096, 16, 1 << 16, 8
    x = to_device(synth.small_stream(P, T, chunk * nch, in_dtype=synth.IN_CI8, seed=77).generate())
    plan = pkg.Plan(P, T, pkg.PFB_IN_CI8, pkg.PFB_WIN_BLACKMAN)
    srv = pkg.Server(hbm_budget_bytes=1 << 30, max_slots=8)
    want = _chunked(srv, plan, x, chunk)
    sid = srv.open_stream(plan)
    out = torch.full((want.shape[0], P), 5.0, dtype=torch.complex64, device="cuda")
    t_before = time.monotonic()
    tks = srv.submit_chunks(sid, x, nch, chunk, out)
    assert len(tks) == nch and len(set(tks)) == nch
    for t in tks:
        assert srv.wait(t, 20000) == pkg.PFB_OK
    t_after = time.monotonic()
    torch.cuda.synchronize()
    assert torch.equal(out, want)
    prev_done = 0.0
    for t in tks:
        ts, td = srv.ticket_times(t)
        assert t_before - 1e-3 <= ts <= td <= t_after + 1e-3
        assert td >= prev_done   # chunks of one stream complete in order
        prev_done = td
    # a too-small output is rejected before anything is submitted past it
    sid2 = srv.open_stream(plan)
    small = torch.empty((3, P), dtype=torch.complex64, device="cuda")
    with pytest.raises(pkg.PFBError) as e:
        srv.submit_chunks(sid2, x, nch, chunk, small)
    assert e.value.status == pkg.PFB_ERR_INVALID
    srv.close_stream(sid)
    assert srv.close() in (pkg.PFB_OK,)
