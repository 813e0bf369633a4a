"""Static checks of the CUDA sources (CPU): every device-side spin wait is bounded, and no kernel
traps on purpose.

- The only `mbarrier.try_wait` is inside `mbar_try_wait` (csrc/tc_ptx.cuh), and the only caller of
  `mbar_try_wait` is `mbar_wait`, whose loop gives up after WAIT_LIMIT cycles and sets the status.
- Every `mbar_wait` call passes the status pointer (three arguments).
- No `__trap()` or PTX `trap`."""
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2011_01400_gb300", "csrc")


def sources():
    files = sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cuh")) +
                   glob.glob(os.path.join(CSRC, "*.h")))
    assert files
    return {os.path.basename(f): open(f).read() for f in files}


def call_args(src, name):
    """Argument lists of every call name(...) in src (balanced parentheses)."""
    out = []
    for m in re.finditer(r"\b%s\s*\(" % re.escape(name), src):
        i, depth, start = m.end(), 1, m.end()
        while depth:
            c = src[i]
            depth += c == "("
            depth -= c == ")"
            i += 1
        out.append(src[start:i - 1])
    return out


def top_level_commas(args):
    depth = n = 0
    for c in args:
        if c in "([{":
            depth += 1
        elif c in ")]}":
            depth -= 1
        elif c == "," and depth == 0:
            n += 1
    return n


def test_try_wait_only_inside_the_bounded_helper():
    src = sources()
    for name, text in src.items():
        if name != "tc_ptx.cuh":
            assert "mbarrier.try_wait" not in text, name
            assert not call_args(text, "mbar_try_wait"), name
    helper = src["tc_ptx.cuh"]
    body = helper[helper.index("bool mbar_wait("):]
    body = body[:body.index("\n}\n")]
    assert "WAIT_LIMIT" in body and "ST_TIMEOUT" in body and "return false" in body


def test_every_wait_passes_the_status():
    n = 0
    for name, text in sources().items():
        for args in call_args(text, "mbar_wait"):
            if args.strip().startswith("uint64_t*"):
                continue                      # the definition
            assert top_level_commas(args) == 2, (name, args)
            n += 1
    assert n > 20


def test_no_trap():
    for name, text in sources().items():
        assert "__trap" not in text, name
        assert not re.search(r"\btrap\s*;", text), name
