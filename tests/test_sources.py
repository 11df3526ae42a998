"""Static checks of the CUDA sources (no GPU): every kernel launched with
programmatic dependent launch waits for the grids before it as its first
statement.  Such a kernel may be scheduled while its predecessor still runs;
a read (or write) of the predecessor's buffers before griddepcontrol.wait
would race with it."""
from __future__ import annotations

import re
from pathlib import Path

CSRC = Path(__file__).resolve().parent.parent / "paper_2603_08499_gb300" / "csrc"


def _sources():
    return {p.name: p.read_text() for p in sorted(CSRC.glob("*.cu"))}


def _kernel_body(src: str, name: str) -> str | None:
    m = re.search(r"__global__[^;{]*?\b" + re.escape(name) + r"\s*\(", src)
    if not m:
        return None
    i, depth = m.end(), 1
    while depth:
        depth += {"(": 1, ")": -1}.get(src[i], 0)
        i += 1
    j = src.index("{", i)
    return src[j + 1:]


def test_pdl_kernels_wait_first():
    srcs = _sources()
    launched = set()
    for text in srcs.values():
        launched |= set(re.findall(r"launch_pdl\(\s*(\w+)", text))
    assert len(launched) >= 15, launched
    for name in sorted(launched):
        bodies = [b for b in (_kernel_body(t, name) for t in srcs.values()) if b is not None]
        assert bodies, f"kernel {name} not found"
        for b in bodies:
            first = [ln.strip() for ln in b.splitlines() if ln.strip()][:2]
            assert first[0] == "pdl_wait();", (name, first)


def test_no_plain_launch_of_pdl_kernels():
    """A kernel that is launched with the attribute anywhere is launched with
    it everywhere in the hot-path files, so no launch site is missed."""
    srcs = _sources()
    launched = set()
    for text in srcs.values():
        launched |= set(re.findall(r"launch_pdl\(\s*(\w+)", text))
    for fname, text in srcs.items():
        for name in launched:
            plain = re.findall(r"\b" + name + r"(?:<[^<>]*>)?<<<", text)
            if fname in ("vbgs_estep_tc.cu", "vbgs_mstep.cu", "vbgs_sort.cu"):
                assert not plain, (fname, name)


def test_pass1_traffic_digest(tmp_path):
    """The benchmark reports pass 1's DRAM traffic from an ncu capture only
    while the kernel's source digest matches the captured one; the digest is
    found (a renamed or moved kernel would silently turn the figure off) and
    differs when the kernel's text changes."""
    import bench
    path = CSRC / "vbgs_estep_tc.cu"
    d = bench.kernel_digest("k_pass1_tc", path)
    assert d is not None and len(d) == 40
    src = path.read_text()
    body = _kernel_body(src, "k_pass1_tc")
    edited = src.replace(body, body.replace("pdl_wait();", "pdl_wait(); ", 1), 1)
    tmp = tmp_path / "edited.cu"
    tmp.write_text(edited)
    assert bench.kernel_digest("k_pass1_tc", tmp) != d
    assert bench.pass1_traffic("bf16x3") is None
