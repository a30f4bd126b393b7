"""The committed ncu / measurement summaries stay reproducible (no GPU): every `python bench.py ...`
command they give parses with bench.py's own argument parser, and each summary names its command."""
import glob
import os
import re
import shlex
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md")) + glob.glob(os.path.join(ROOT, "profiles", "*.txt")))


def bench_commands(path):
    """The argument lists of the `python bench.py` invocations in a summary (plain or under ncu)."""
    out = []
    for line in open(path, encoding="utf-8"):
        m = re.search(r"python bench\.py(.*)$", line)
        if not m:
            continue
        tail = re.sub(r"\(.*?\)\s*$", "", m.group(1)).strip()   # a trailing "(another call)" note
        tail = tail.split(">")[0].split("&&")[0].strip()
        out.append(shlex.split(tail))
    return out


def test_there_are_summaries():
    assert PROFILES, "profiles/ holds no summaries"


@pytest.mark.parametrize("path", PROFILES, ids=[os.path.basename(p) for p in PROFILES])
def test_summary_commands_parse_with_bench(path):
    sys.path.insert(0, ROOT)
    import bench

    cmds = bench_commands(path)
    assert cmds, f"{os.path.basename(path)} gives no bench.py command"
    parser = bench.build_parser()
    for argv in cmds:
        parser.parse_args(argv)


@pytest.mark.parametrize("path", PROFILES, ids=[os.path.basename(p) for p in PROFILES])
def test_summary_is_short_text(path):
    assert os.path.getsize(path) < 16 * 1024
    text = open(path, encoding="utf-8").read()
    assert "_work/" not in text
