"""Static checks of the CUDA sources (CPU).

Every kernel is launched through gs::launch, which allows programmatic
dependent launch: a kernel may be scheduled before its predecessor on the
stream has finished, so it must wait for it (kernel_prologue) before it
touches memory (gs::launch_serial, an ordinary launch, is kept for the
kernels measured slower with it). These checks keep that invariant: no kernel
launched with the triple-chevron syntax, and every __global__ function's
first statement is the prologue."""
import glob
import os
import re

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2412_13547_b300", "csrc")
SOURCES = sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cuh")))


def _strip_comments(s):
    s = re.sub(r"/\*.*?\*/", "", s, flags=re.S)
    return re.sub(r"//[^\n]*", "", s)


def test_sources_found():
    assert len(SOURCES) >= 7


def test_no_chevron_launches():
    for f in SOURCES:
        s = _strip_comments(open(f).read())
        assert "<<<" not in s, f"{os.path.basename(f)} launches a kernel without gs::launch"


def test_every_kernel_starts_with_the_prologue():
    n = 0
    for f in SOURCES:
        s = _strip_comments(open(f).read())
        for m in re.finditer(r"__global__\s+void\b", s):
            body = s.index("{", m.end())
            # the parameter list ends before the body; no ';' in between (a declaration)
            assert ";" not in s[m.end():body], f"{os.path.basename(f)}: kernel declaration without a body"
            first = s[body + 1:].lstrip()
            assert first.startswith("kernel_prologue();"), \
                f"{os.path.basename(f)}: kernel at offset {m.start()} does not start with kernel_prologue()"
            n += 1
    assert n >= 40
