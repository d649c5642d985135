"""The serving loop on the GPU: every request's result is bitwise the same alone and in
the concurrent mix, matches the oracle within the FP32-mixed tolerance, requests too
large for the arena are rejected, and Poisson arrivals produce latency statistics."""

import numpy as np
import pytest
import torch

import oracle
import workloads
from gpu_util import TOL, rel_err
import paper_1607_04245_gb300 as fem
from paper_1607_04245_gb300.serving import (GpuExecutor, Scheduler, footprint, make_request, make_selftest_request,
                                            poisson_arrivals)

pytestmark = pytest.mark.gpu


def _stream(n, seed, max_cells, prec="mixed"):
    specs = workloads.cases.serving_specs(n, seed=seed, min_cells=1000, max_cells=max_cells)
    cases = [workloads.cases.serving_case(s) for s in specs]
    return cases, [make_request(s["rid"], c, s["kind"], prec) for s, c in zip(specs, cases)]


def test_mix_equals_alone_and_matches_oracle():
    cases, mix = _stream(48, seed=11, max_cells=60000)
    biggest = max(footprint(r) for r in mix)
    ex = GpuExecutor(capacity=3 * biggest, n_slots=6)  # memory, not slots, limits admission
    st = Scheduler(ex).run(mix)
    assert st.n_done == len(mix) and st.n_rejected == 0
    assert st.max_inflight >= 2  # work really overlapped
    _, alone = _stream(48, seed=11, max_cells=60000)
    ex1 = GpuExecutor(capacity=2 * biggest, n_slots=1)
    for r in alone:
        Scheduler(ex1).run([r])
    for a, b in zip(mix, alone):
        assert a.result.keys() == b.result.keys()
        for k in a.result:
            assert torch.equal(a.result[k], b.result[k]), (a.rid, k)
    for c, r in zip(cases, mix):
        c32 = c.rounded_to_f32()
        if r.kind == "residual":
            assert rel_err(r.result["out"], oracle.residual_for(c32)) <= TOL["mixed"]
        else:
            rK, ru = oracle.adjoint_for(c32)
            assert rel_err(r.result["dK"], rK) <= TOL["mixed"] and rel_err(r.result["du"], ru) <= TOL["mixed"]


def test_too_large_request_is_rejected():
    cases, reqs = _stream(6, seed=5, max_cells=20000)
    small = min(footprint(r) for r in reqs)
    ex = GpuExecutor(capacity=small + 4096, n_slots=2, nvtx=True)  # the NVTX ranges cost nothing unprofiled
    st = Scheduler(ex).run(reqs)
    assert st.n_rejected >= 1
    assert st.n_done + st.n_rejected == len(reqs)
    assert all(r.status in ("done", "rejected") for r in reqs)


def test_poisson_arrivals_latency():
    cases, reqs = _stream(60, seed=3, max_cells=100000)
    t = poisson_arrivals(len(reqs), rate=400.0, seed=9)
    for r, a in zip(reqs, t):
        r.arrival = float(a)
    ex = GpuExecutor(capacity=1 << 30, n_slots=8)
    st = Scheduler(ex).run(reqs, arrival_rate=400.0)
    assert st.n_done == len(reqs)
    assert 0 < st.p50_ms <= st.p99_ms
    assert st.makespan_s >= t[-1]
    assert all(r.t_done > r.t_arrive for r in reqs)


def test_failed_requests_are_reported_and_isolated():
    """A request whose mesh is invalid (an out-of-range vertex id) and a self-test request
    whose bounded wait gives up come back failed with their reason, read from their own
    error words; the requests served beside them are unaffected (bitwise equal to their
    results alone) and the device-wide error word stays clear."""
    _, mix = _stream(16, seed=21, max_cells=30000)
    victim = next(r for r in mix if r.kind == "residual")
    victim.host["conn"][0, 3] = victim.n_verts + 5  # a view into the request's pinned input block
    probe = make_selftest_request(999, arrival=0.0)
    ex = GpuExecutor(capacity=1 << 30, n_slots=4)
    assert fem.fem_device_error() == 0
    st = Scheduler(ex).run(mix + [probe])
    assert st.n_failed == 2 and st.n_done == len(mix) - 1
    assert victim.status == "failed" and "bad mesh" in victim.error
    assert probe.status == "failed" and "timeout" in probe.error
    assert fem.fem_device_error() == 0
    _, alone = _stream(16, seed=21, max_cells=30000)
    ex1 = GpuExecutor(capacity=1 << 30, n_slots=1)
    for a, b in zip(mix, alone):
        if a is victim:
            continue
        Scheduler(ex1).run([b])
        assert a.status == "done" and b.status == "done"
        for k in a.result:
            assert torch.equal(a.result[k], b.result[k]), (a.rid, k)


def test_native_loop_equals_python_loop_and_alone():
    """fem_serve_run (the whole stream in one native call) serves every request with the
    same results, bitwise, as the Python scheduler and as the request alone; memory, not
    slots, limits admission so backfill and overlap both happen."""
    from paper_1607_04245_gb300.serving import NativeScheduler

    _, mix = _stream(40, seed=13, max_cells=60000)
    biggest = max(footprint(r) for r in mix)
    ex = GpuExecutor(capacity=3 * biggest, n_slots=6)
    st = NativeScheduler(ex).run(mix)
    assert st.n_done == len(mix) and st.n_rejected == 0 and st.n_failed == 0
    assert st.max_inflight >= 2
    assert all(r.t_arrive <= r.t_admit <= r.t_done for r in mix)
    _, ref = _stream(40, seed=13, max_cells=60000)
    Scheduler(GpuExecutor(capacity=3 * biggest, n_slots=6)).run(ref)
    for a, b in zip(mix, ref):
        for k in a.result:
            assert torch.equal(a.result[k], b.result[k]), (a.rid, k)
    # a second pass over the same requests (status words re-zeroed by the loop)
    st2 = NativeScheduler(ex).run(mix)
    assert st2.n_done == len(mix)


def test_native_loop_failures_rejections_and_refusals():
    """In the native loop: a bad-mesh request and a self-test request fail with their bits,
    a request larger than the arena is rejected on arrival, a descriptor the launcher
    refuses (an array outside its block) fails alone, and the rest are bitwise the same as
    when served alone."""
    from paper_1607_04245_gb300.serving import NativeScheduler, SERVE_SLOTS

    _, mix = _stream(14, seed=23, max_cells=30000)
    victim = next(r for r in mix if r.kind == "residual")
    victim.host["conn"][0, 2] = victim.n_verts + 3
    refused = next(r for r in mix if r.kind == "residual" and r is not victim)
    refused.desc.offset[SERVE_SLOTS["out"]] = footprint(refused)  # its output array past the block's end
    probe = make_selftest_request(998)
    spec = workloads.cases.serving_specs(1, seed=4, min_cells=400000, max_cells=500000)[0]
    huge = make_request(997, workloads.cases.serving_case(spec), spec["kind"], "mixed")
    cap = max(footprint(r) for r in mix) * 2
    assert footprint(huge) > cap
    ex = GpuExecutor(capacity=cap, n_slots=4)
    reqs = mix + [probe, huge]
    assert fem.fem_device_error() == 0
    st = NativeScheduler(ex).run(reqs)
    assert victim.status == "failed" and "bad mesh" in victim.error
    assert probe.status == "failed" and "timeout" in probe.error
    assert refused.status == "failed" and "refused" in refused.error
    assert huge.status == "rejected" and st.n_rejected == 1
    assert st.n_failed == 3 and st.n_done == len(mix) - 2
    assert fem.fem_device_error() == 0
    _, alone = _stream(14, seed=23, max_cells=30000)
    ex1 = GpuExecutor(capacity=1 << 30, n_slots=1)
    for a, b in zip(mix, alone):
        if a is victim or a is refused:
            continue
        Scheduler(ex1).run([b])
        assert a.status == "done"
        for k in a.result:
            assert torch.equal(a.result[k], b.result[k]), (a.rid, k)


def test_native_loop_poisson_arrivals():
    from paper_1607_04245_gb300.serving import NativeScheduler

    _, reqs = _stream(60, seed=3, max_cells=100000)
    t = poisson_arrivals(len(reqs), rate=500.0, seed=9)
    for r, a in zip(reqs, t):
        r.arrival = float(a)
    ex = GpuExecutor(capacity=1 << 30, n_slots=8)
    st = NativeScheduler(ex).run(reqs, arrival_rate=500.0)
    assert st.n_done == len(reqs)
    assert 0 < st.p50_ms <= st.p99_ms
    assert st.makespan_s >= t[-1]
    t0 = min(r.t_arrive for r in reqs)
    # arrivals are honoured: nothing is admitted before it arrives
    for r in reqs:
        assert abs((r.t_arrive - t0) - (r.arrival - t[0])) < 1e-6
        assert r.t_admit >= r.t_arrive - 1e-9
