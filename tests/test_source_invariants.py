"""Static checks of the CUDA sources (no GPU): rules that a kernel launch
relies on but the compiler cannot enforce.

A kernel launched as a programmatic dependent launch may start while the
previous kernel of its stream is still running; it is only safe if its
first statement waits for that kernel (griddepcontrol.wait).  Every kernel
that some launch site may launch that way must therefore begin with
griddep_wait().
"""
import os
import re

import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_1402_3281_gb300", "csrc")


def _sources():
    return {f: open(os.path.join(CSRC, f)).read() for f in sorted(os.listdir(CSRC))
            if f.endswith((".cu", ".cuh"))}


def _pdl_launched(src):
    """Kernels passed to launch_k with a flag that is not the literal false."""
    names = set()
    for m in re.finditer(r"launch_k\(\s*([^,]+?)\s*,\s*([A-Za-z_][A-Za-z_0-9]*)", src):
        if m.group(1).startswith("bool "):        # the helper's own definition
            continue
        if m.group(1) != "false":
            names.add(m.group(2))
    return names


def _first_statement(src, kernel):
    m = re.search(r"__global__\s+void[^{;]*?\b" + kernel + r"\s*\([^)]*\)\s*\{\s*([^;]*;)", src,
                  re.S)
    return m.group(1).strip() if m else None


def test_some_kernels_are_launched_programmatically():
    launched = set()
    for src in _sources().values():
        launched |= _pdl_launched(src)
    assert {"k_bucket_count", "k_bucket_scatter", "k_round_cond"} <= launched


def _kernels_calling(src, callee):
    """__global__ functions whose body calls `callee` (directly)."""
    out = set()
    for m in re.finditer(r"__global__\s+void[^{;]*?\b(k_[A-Za-z_0-9]+)\s*\(", src):
        start = src.index("{", m.end())
        depth, i = 0, start
        while True:
            if src[i] == "{":
                depth += 1
            elif src[i] == "}":
                depth -= 1
                if depth == 0:
                    break
            i += 1
        if re.search(r"\b" + callee + r"\s*\(", src[start:i]):
            out.add(m.group(1))
    return out


def test_grid_barriers_only_in_cooperative_launches():
    """A grid-wide barrier needs every CTA resident at once: a kernel that
    calls grid_sync must be launched with launch_coop and never with a plain
    or programmatic launch."""
    srcs = _sources()
    users = set()
    for src in srcs.values():
        users |= _kernels_calling(src, "grid_sync")
    assert "k_admit" in users
    coop = set()
    for src in srcs.values():
        coop |= set(re.findall(r"launch_coop\(\s*([A-Za-z_][A-Za-z_0-9]*)", src))
        plain = set(re.findall(r"\b(k_[A-Za-z_0-9]+)\s*<<<", src)) | _pdl_launched(src)
        plain |= {m.group(1) for m in re.finditer(
            r"launch_k\(\s*false\s*,\s*([A-Za-z_][A-Za-z_0-9]*)", src)}
        assert not (users & plain), users & plain
    assert users <= coop, users - coop


@pytest.mark.parametrize("fname", sorted(_sources()))
def test_programmatic_launches_wait_first(fname):
    srcs = _sources()
    for kernel in sorted(_pdl_launched(srcs[fname])):
        defs = [f for f, s in srcs.items() if _first_statement(s, kernel) is not None]
        assert defs, f"{kernel}: definition not found"
        for f in defs:
            assert _first_statement(srcs[f], kernel) == "griddep_wait();", (f, kernel)


def test_helper_waits_with_griddepcontrol():
    src = _sources()["common.cuh"]
    body = re.search(r"void griddep_wait\(\)\s*\{(.*?)\}", src, re.S).group(1)
    assert "griddepcontrol.wait" in body
