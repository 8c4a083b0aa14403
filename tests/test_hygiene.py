"""Repository rules that a later change could break silently (no GPU)."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SOURCE_DIRS = ["paper_2608_25203_b300", "include", "oracle", "tests"]
SOURCE_FILES = ["bench.py", "__graft_entry__.py"]
EXT = (".py", ".cu", ".cuh", ".h", ".c", ".cpp")


def _sources():
    for d in SOURCE_DIRS:
        for dirpath, _, files in os.walk(os.path.join(ROOT, d)):
            if "__pycache__" in dirpath:
                continue
            for f in files:
                if f.endswith(EXT):
                    yield os.path.join(dirpath, f)
    for f in SOURCE_FILES:
        yield os.path.join(ROOT, f)


def test_no_batched_memcpy_calls():
    # the batched host/device copy entry points are closed on the GPU pool: copies go one
    # cudaMemcpyAsync at a time
    pat = re.compile(r"Memcpy(3D)?" + "Batch" + r"Async")
    bad = [p for p in _sources() if pat.search(open(p, errors="replace").read())]
    assert not bad, bad


def test_profile_commands_leave_clocks_alone():
    pdir = os.path.join(ROOT, "profiles")
    for f in sorted(os.listdir(pdir)):
        for line in open(os.path.join(pdir, f)):
            if re.match(r"\s*ncu\s", line) and " -i " not in line:
                assert "--clock-control none" in line, (f, line.strip())


def test_nothing_committed_reads_the_scratch_folder():
    bad = []
    for p in _sources():
        if os.path.abspath(p) == os.path.abspath(__file__):
            continue
        txt = open(p, errors="replace").read()
        if re.search(r"[\"'/]_work[/\"']|import _work|from _work", txt):
            bad.append(p)
    assert not bad, bad
