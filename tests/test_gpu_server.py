"""Serving: requests of mixed sizes and step counts admitted by HBM budget,
batched as they arrive; each result equals the request run alone (bit for
bit) and matches the FP64 oracle (max |dpsi| <= 1e-5 max|psi| up to 10
steps, <= 1e-4 beyond).  Failure handling is exercised on the host: over-budget submits,
timeouts, cancellation and an injected allocation failure."""
import threading

import numpy as np
import pytest

import gen.fields as F
from gpu_helpers import rel_err, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mp():
    import __graft_entry__ as g
    g.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1507_01265_gb300 as mp
    return mp


def _requests(n, seed=5):
    st = F.Stream(seed)
    out = []
    for i in range(n):
        nx = 4 * st.log_uniform_int(8, 40) + (0 if i % 3 else 1)  # some nx % 4 != 0
        ny = st.log_uniform_int(8, 90)
        nz = st.log_uniform_int(4, 24)
        per = (1, 1, 0) if i % 2 else (1, 1, 1)
        f = F.rotation_blobs(nx=nx, ny=ny, nz=nz, max_c=st.scalar(0.1, 0.5), nblobs=2,
                             nsteps=int(st.scalar(1, 30)), seed=100 + i, periodic=per)
        out.append(f)
    return out


def test_results_equal_alone_in_the_mix(mp):
    fs = _requests(24)
    outs = [f.psi.copy() for f in fs]
    with mp.Server(hbm_budget_bytes=64 << 20, chunk_steps=4) as srv:
        tickets = []
        # submit from two threads while earlier requests are already running
        def worker(idx):
            for i in idx:
                f = fs[i]
                tickets.append((i, srv.submit(f.h, outs[i], f.u1, f.u2, f.u3, f.nsteps, periodic=f.periodic)))
        th = [threading.Thread(target=worker, args=(range(k, len(fs), 2),)) for k in (0, 1)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        for i, tk in tickets:
            srv.wait(tk, timeout_ms=60000)
            assert srv.poll(tk) == mp._lib.REQ_DONE
            t0, t1, t2 = srv.times(tk)
            assert t0 <= t1 <= t2
        st = srv.stats()
        assert st["completed"] == len(fs) and st["resident"] == 0 and st["admitted_bytes"] == 0
    for f, o in zip(fs, outs):
        got = o.astype(np.float64)
        assert np.array_equal(got, run_gpu(f, f.nsteps, tile=(32, 24))), f.name
        tol = 1e-5 if f.nsteps <= 10 else 1e-4
        assert rel_err(got, run_oracle(f, f.nsteps)) <= tol, f.name


def test_budget_refusal_timeout_cancel(mp):
    f = F.rotation_blobs(nx=64, ny=64, nz=16, seed=3)
    need = 6 * f.ncells * 4
    with mp.Server(hbm_budget_bytes=need, max_queued=0, chunk_steps=2) as srv:
        a = f.psi.copy()
        # long enough (several seconds) to still be resident for the checks below
        ta = srv.submit(f.h, a, f.u1, f.u2, f.u3, 200000, periodic=f.periodic)
        with pytest.raises(mp.MpdataError) as e:  # budget reserved by the first request
            srv.submit(f.h, f.psi.copy(), f.u1, f.u2, f.u3, 1, periodic=f.periodic)
        assert e.value.code == mp._lib.MPDATA_EBUSY
        with pytest.raises(mp.MpdataError) as e:
            srv.wait(ta, timeout_ms=0)
        assert e.value.code == mp._lib.MPDATA_ETIMEDOUT
        srv.cancel(ta)
        with pytest.raises(mp.MpdataError) as e:
            srv.wait(ta, timeout_ms=60000)
        assert e.value.code == mp._lib.MPDATA_ECANCELED
        # budget is free again
        b = f.psi.copy()
        tb = srv.submit(f.h, b, f.u1, f.u2, f.u3, 3, periodic=f.periodic)
        srv.wait(tb, timeout_ms=60000)
        assert np.array_equal(b.astype(np.float64), run_gpu(f, 3, tile=(32, 24)))
        with pytest.raises(mp.MpdataError) as e:
            srv.poll(999999)
        assert e.value.code == mp._lib.MPDATA_ENOENT
        with pytest.raises(mp.MpdataError) as e:  # larger than the whole budget
            g = F.rotation_blobs(nx=128, ny=64, nz=16, seed=4)
            srv.submit(g.h, g.psi.copy(), g.u1, g.u2, g.u3, 1)
        assert e.value.code == mp._lib.MPDATA_EINVAL


def test_injected_allocation_failure(mp):
    fs = _requests(4, seed=9)
    outs = [f.psi.copy() for f in fs]
    with mp.Server(hbm_budget_bytes=256 << 20, inject_alloc_failure=2) as srv:
        ts = [srv.submit(f.h, o, f.u1, f.u2, f.u3, f.nsteps, periodic=f.periodic) for f, o in zip(fs, outs)]
        codes = []
        for t in ts:
            try:
                srv.wait(t, timeout_ms=60000)
                codes.append(0)
            except mp.MpdataError as e:
                codes.append(e.code)
    assert codes == [0, mp._lib.MPDATA_ENOMEM, 0, mp._lib.MPDATA_ENOMEM]
    for i in (0, 2):
        assert np.array_equal(outs[i].astype(np.float64), run_gpu(fs[i], fs[i].nsteps, tile=(32, 24)))


def test_finished_requests_are_retired(mp):
    """A server that runs on holds a bounded number of finished requests: the
    oldest are retired beyond retain_finished, mpdata_release forgets one at
    once, and a request still running cannot be released."""
    f = F.rotation_blobs(nx=16, ny=8, nz=4, nblobs=1, seed=6)
    keep = 8
    with mp.Server(hbm_budget_bytes=64 << 20, retain_finished=keep) as srv:
        tickets = []
        for i in range(120):
            tickets.append(srv.submit(f.h, f.psi.copy(), f.u1, f.u2, f.u3, 2, periodic=f.periodic))
            if i % 10 == 9:
                for t in tickets[-10:]:
                    _wait_or_retired(mp, srv, t)
                assert srv.retained() <= keep
        assert srv.retained() <= keep
        with pytest.raises(mp.MpdataError) as e:   # retired long ago
            srv.poll(tickets[0])
        assert e.value.code == mp._lib.MPDATA_ENOENT
        last = tickets[-1]
        assert srv.poll(last) == mp._lib.REQ_DONE
        srv.release(last)
        with pytest.raises(mp.MpdataError) as e:
            srv.times(last)
        assert e.value.code == mp._lib.MPDATA_ENOENT
        busy = srv.submit(f.h, f.psi.copy(), f.u1, f.u2, f.u3, 100000, periodic=f.periodic)
        with pytest.raises(mp.MpdataError) as e:   # still running
            srv.release(busy)
        assert e.value.code == mp._lib.MPDATA_EBUSY
        srv.cancel(busy)
        with pytest.raises(mp.MpdataError):
            srv.wait(busy, timeout_ms=60000)
        srv.release(busy)
        assert srv.retained() <= keep


def _wait_or_retired(mp, srv, ticket):
    """Wait for a request; ENOENT means it finished and was retired already."""
    try:
        srv.wait(ticket, timeout_ms=60000)
    except mp.MpdataError as e:
        assert e.code == mp._lib.MPDATA_ENOENT


def test_destroy_releases_blocked_waiters(mp):
    """Destroying a server while another thread is blocked in mpdata_wait on
    a running request cancels it and returns that wait (ECANCELED) before
    anything is freed."""
    f = F.rotation_blobs(nx=64, ny=64, nz=16, nblobs=1, seed=8)
    srv = mp.Server(hbm_budget_bytes=64 << 20)
    t = srv.submit(f.h, f.psi.copy(), f.u1, f.u2, f.u3, 10 ** 7, periodic=f.periodic)
    codes = []
    started = threading.Event()

    def waiter():
        started.set()
        try:
            srv.wait(t)
            codes.append(0)
        except mp.MpdataError as e:
            codes.append(e.code)

    th = threading.Thread(target=waiter)
    th.start()
    started.wait()
    import time
    time.sleep(0.2)  # the waiter is inside mpdata_wait
    srv.close()
    th.join(timeout=60)
    assert not th.is_alive()
    assert codes == [mp._lib.MPDATA_ECANCELED]


def test_more_resident_requests_than_direct_runs(mp):
    """Ticks normally pass their grid table in the kernel parameters (up to
    320 requests per kernel variant); with more requests resident the tick
    uploads the table and runs the general batched kernel.  Either way each
    result is the request's bits alone."""
    st = F.Stream(13)
    fs = []
    for i in range(360):
        nx, ny, nz = 8 + 4 * int(st.scalar(0, 3)), 8 + int(st.scalar(0, 5)), 4
        fs.append(F.rotation_blobs(nx=nx, ny=ny, nz=nz, max_c=0.3, nblobs=1, nsteps=40, seed=500 + i,
                                   periodic=(1, 1, 0)))
    outs = [f.psi.copy() for f in fs]
    with mp.Server(hbm_budget_bytes=256 << 20, max_active=512, chunk_steps=2) as srv:
        tickets = [srv.submit(f.h, o, f.u1, f.u2, f.u3, f.nsteps, periodic=f.periodic) for f, o in zip(fs, outs)]
        for t in tickets:
            srv.wait(t, timeout_ms=120000)
    for f, o in zip(fs[::7], outs[::7]):
        assert np.array_equal(o.astype(np.float64), run_gpu(f, f.nsteps, tile=(32, 24))), f.name
