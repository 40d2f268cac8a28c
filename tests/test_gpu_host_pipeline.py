"""Pipelined host solves (mpdata_host_submit / mpdata_host_wait): each solve's
result must be bit-identical to the same solve run alone, whatever the
slot it took, the solves in flight beside it and the order of the waits;
one result is also checked against the FP64 oracle."""
import numpy as np
import pytest

from gpu_helpers import rand_problem, rel_err, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

SHAPE = (10, 36, 40)  # nz, ny, nx: nx % 4 == 0, several tiles, ragged tail in y


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _pinned(f):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (f.h, f.psi, f.u1, f.u2, f.u3)]


def _alone(f, nsteps):
    return run_gpu(f, nsteps, tile=(32, 24)).astype(np.float32)


def test_pipeline_matches_solves_alone():
    import paper_1507_01265_gb300 as mp
    probs = [rand_problem(SHAPE, 700 + i) for i in range(5)]
    nsteps = [3, 4, 0, 5, 2]
    with mp.Solver(40, 36, 10, periodic=(1, 1, 1), tile=(32, 24)) as s:
        host = [_pinned(f) for f in probs]
        outs = [a[1].clone().pin_memory() for a in host]
        tickets = [s.submit_host(*a, n, psi_out=o) for a, n, o in zip(host, nsteps, outs)]
        assert tickets == [1, 2, 3, 4, 5]
        s.wait_host(tickets[-1])
        for f, n, o, a in zip(probs, nsteps, outs, host):
            assert np.array_equal(o.numpy(), _alone(f, n))
            assert np.array_equal(a[1].numpy(), f.psi)  # psi_in untouched when psi_out differs


def test_pipeline_in_place_and_out_of_order_waits():
    import paper_1507_01265_gb300 as mp
    from paper_1507_01265_gb300 import MpdataError
    probs = [rand_problem(SHAPE, 720 + i, periodic=(0, 1, 0)) for i in range(4)]
    with mp.Solver(40, 36, 10, periodic=(0, 1, 0), tile=(32, 24)) as s:
        host = [_pinned(f) for f in probs]
        tickets = [s.submit_host(*a, 6) for a in host]  # psi_out = psi_in
        s.wait_host(tickets[2])
        for f, a in zip(probs[:3], host[:3]):
            assert np.array_equal(a[1].numpy(), _alone(f, 6))
        s.wait_host(tickets[0])  # already done: returns at once
        s.wait_host(tickets[3])
        assert np.array_equal(host[3][1].numpy(), _alone(probs[3], 6))
        for bad in (0, tickets[-1] + 1):
            with pytest.raises(MpdataError) as ei:
                s.wait_host(bad)
            assert ei.value.code == mp._lib.MPDATA_ENOENT


def test_pipeline_more_tickets_than_the_ring():
    """20 solves in flight (the per-ticket event ring holds 16): every wait,
    including one for a ticket whose ring entry a later solve re-recorded,
    returns only after that solve's result has landed."""
    import paper_1507_01265_gb300 as mp
    probs = [rand_problem(SHAPE, 740 + i) for i in range(20)]
    with mp.Solver(40, 36, 10, periodic=(1, 1, 1), tile=(32, 24)) as s:
        host = [_pinned(f) for f in probs]
        tickets = [s.submit_host(*a, 2 + (i % 3)) for i, a in enumerate(host)]
        s.wait_host(tickets[1])  # its ring entry was re-recorded by ticket 18
        assert np.array_equal(host[1][1].numpy(), _alone(probs[1], 3))
        s.wait_host(tickets[-1])
        for i, (f, a) in enumerate(zip(probs, host)):
            assert np.array_equal(a[1].numpy(), _alone(f, 2 + (i % 3)))


def test_pipeline_interleaved_with_solve_host_and_pageable_arrays():
    """solve_host shares slot 0 and the scratch buffer with the pipeline: it
    must wait for the solves in flight.  Pageable numpy arrays give the same
    results (the copies then block the host)."""
    import paper_1507_01265_gb300 as mp
    probs = [rand_problem(SHAPE, 760 + i) for i in range(3)]
    with mp.Solver(40, 36, 10, periodic=(1, 1, 1), tile=(32, 24)) as s:
        host = [_pinned(f) for f in probs[:2]]
        t = [s.submit_host(*a, 7) for a in host]
        sync = [np.array(a, copy=True) for a in (probs[2].h, probs[2].psi, probs[2].u1, probs[2].u2, probs[2].u3)]
        s.solve_host(*sync, 7)
        pageable = [np.array(a, copy=True) for a in (probs[0].h, probs[0].psi, probs[0].u1,
                                                   probs[0].u2, probs[0].u3)]
        t3 = s.submit_host(*pageable, 7)
        s.wait_host(t3)
        assert t3 == t[-1] + 1
        assert np.array_equal(host[0][1].numpy(), _alone(probs[0], 7))
        assert np.array_equal(host[1][1].numpy(), _alone(probs[1], 7))
        assert np.array_equal(sync[1], _alone(probs[2], 7))
        assert np.array_equal(pageable[1], _alone(probs[0], 7))


def test_pipeline_against_oracle_and_f64():
    import paper_1507_01265_gb300 as mp
    f = rand_problem(SHAPE, 780)
    want = run_oracle(f, 10)
    with mp.Solver(40, 36, 10, periodic=(1, 1, 1)) as s:
        a = _pinned(f)
        s.wait_host(s.submit_host(*a, 10))
        assert rel_err(a[1].numpy().astype(np.float64), want) <= 1e-5
    with mp.Solver(40, 36, 10, periodic=(1, 1, 1), dtype="f64") as s:
        a = [np.array(x, dtype=np.float64) for x in (f.h, f.psi, f.u1, f.u2, f.u3)]
        s.wait_host(s.submit_host(*a, 10))
        assert rel_err(a[1], want) <= 1e-12


def test_pipeline_argument_errors():
    import paper_1507_01265_gb300 as mp
    from paper_1507_01265_gb300 import MpdataError
    f = rand_problem(SHAPE, 790)
    with mp.Solver(40, 36, 10, periodic=(1, 1, 1)) as s:
        a = _pinned(f)
        with pytest.raises(MpdataError) as ei:
            s.submit_host(*a, -1)
        assert ei.value.code == mp._lib.MPDATA_EINVAL
        with pytest.raises(ValueError):
            s.submit_host(*a, 1, psi_out=np.zeros(5, np.float32))
        with pytest.raises(MpdataError) as ei:
            s.wait_host(1)  # nothing issued yet
        assert ei.value.code == mp._lib.MPDATA_ENOENT
