"""Every kernel that the library launches overlapped with the kernel before it
(launch_overlapped: programmatic dependent launch) must wait for that kernel
(griddepcontrol.wait, pdl_wait()) before its first global memory access: a source check,
no GPU needed. It finds each launch_overlapped call, resolves the launched kernel (a
direct template name or the `auto k = ...` it was bound to) and asserts that the kernel's
body opens with pdl_wait()."""

import os
import re

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1607_04245_gb300", "csrc")


def _sources():
    out = {}
    for f in sorted(os.listdir(CSRC)):
        if f.endswith((".cu", ".cuh")):
            out[f] = open(os.path.join(CSRC, f)).read()
    return out


def _kernel_bodies(srcs):
    """name -> list of the first statements of every __global__ definition of that name"""
    bodies = {}
    for text in srcs.values():
        for m in re.finditer(r"__global__\s+void\s+(?:__launch_bounds__\((?:[^()]|\([^()]*\))*\)\s*)?(\w+)\s*\(",
                             text):
            name = m.group(1)
            brace = text.index("{", m.end())
            first = text[brace + 1:brace + 600].strip()
            # compile-time checks and comments come first and touch no memory
            while first.startswith(("static_assert(", "//")):
                first = first[first.index(";" if first.startswith("static") else "\n") + 1:].strip()
            bodies.setdefault(name, []).append(first)
    return bodies


def _launched_kernels(srcs):
    """(file, kernel name) for every launch_overlapped call outside the helper's definition"""
    found = []
    for f, text in srcs.items():
        lines = text.split("\n")
        bound = None
        for ln in lines:
            mk = re.match(r"\s*auto k = (.*);", ln)
            if mk:
                bound = mk.group(1)
            mc = re.search(r"launch_overlapped\(\s*([^,]+),", ln)
            if not mc or "cudaError_t launch_overlapped" in ln:
                continue
            expr = mc.group(1).strip()
            if expr == "k":
                assert bound is not None, (f, ln)
                expr = bound
            names = set(re.findall(r"\b(\w+_kernel)\b", expr))
            assert names, (f, ln)
            found.extend((f, n) for n in names)
    return found


def test_every_overlapped_kernel_waits_first():
    srcs = _sources()
    bodies = _kernel_bodies(srcs)
    launched = _launched_kernels(srcs)
    assert len({n for _, n in launched}) >= 12  # the integration, elasticity, DF and gather kernels
    for f, name in launched:
        assert name in bodies, (f, name)
        for first in bodies[name]:
            assert first.startswith("pdl_wait();"), (f, name, first[:80])


def test_kernels_that_trigger_also_wait():
    """pdl_trigger() only ever follows pdl_wait() at the top of a kernel."""
    for name, firsts in _kernel_bodies(_sources()).items():
        for first in firsts:
            if "pdl_trigger()" in first[:200]:
                assert first.startswith("pdl_wait();"), name


def test_run_time_compiled_kernel_waits_first():
    """The kernel that fem_integrate_pointwise generates (launched overlapped too) opens
    with the same wait, written as inline PTX in its source text."""
    firsts = _kernel_bodies(_sources())["fem_pointwise_kernel"]
    assert firsts and all(f.startswith('asm volatile("griddepcontrol.wait;"') for f in firsts)
