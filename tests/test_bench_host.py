"""Host-side pieces of bench.py that decide what a benchmark line claims."""
import os
import re

import bench


def _closure(tu):
    csrc = os.path.join(os.path.dirname(bench.__file__), "paper_2504_09820_gb300", "csrc")
    seen, todo = set(), [tu]
    while todo:
        f = todo.pop()
        if f in seen or not os.path.exists(os.path.join(csrc, f)):
            continue
        seen.add(f)
        todo += re.findall(r'^#include "([^"/]+)"', open(os.path.join(csrc, f)).read(), re.M)
    return seen


def test_traffic_is_keyed_by_the_head_kernel_sources():
    """The measured DRAM traffic in the roofline object belongs to the head
    kernel's translation unit; the hash covers exactly that file and the csrc
    headers it includes, so an edit elsewhere (another kernel) keeps it and an
    edit of the head kernel drops it to null."""
    files = _closure("detect_tc_k64.cu")
    assert {"detect_tc_k64.cu", "detect_tc_impl.cuh", "cg_warp.cuh", "tc_pipeline.cuh"} <= files
    assert "solve_tc_impl.cuh" not in files and "gram_tc128.cu" not in files
    h = bench.kernel_source_hash()
    assert re.fullmatch(r"[0-9a-f]{12}", h)
    assert bench.kernel_source_hash("detect_tc_k32.cu") != h


def test_algorithmic_bytes_of_one_detection():
    """Read H (N K complex64) and y (N complex64) once; write x_hat (K complex64),
    labels (K bytes), rel_res (8 bytes) and status (4 bytes)."""
    assert bench.bytes_per_detection(256, 64) == 256 * 64 * 8 + 256 * 8 + 64 * 8 + 64 + 8 + 4 == 133708
