"""The committed ncu summaries against the committed kernel: the step kernel's
summary must have been taken on the current kernel sources (the benchmark
takes its DRAM traffic and instruction count from it only then), its figures
must parse, and the traffic it records must sit near the algorithmic bytes of
a launch (600 B per float32 cell, 448 B per float16-deviation cell of the
1024 x 1024 capture); every summary names the command that made it."""
import glob
import os
import re
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

CELLS = 1024 * 1024


def test_step_kernel_summary_matches_the_kernel_sources():
    text = open(bench.PROFILE).read()
    m = re.search(r"kernel_sources_sha:\s*([0-9a-f]+)", text)
    assert m and m.group(1) == bench.kernel_sha(), "re-capture profiles/step_kernel_current_sheet_1024.md"
    for prec, bytes_per_cell in (("fp32", 600), ("fp16", 448)):
        traffic = bench.profiled_traffic(prec)
        instr = bench.profiled_instructions(prec)
        assert traffic is not None and instr is not None, prec
        assert 0.8 < traffic / (bytes_per_cell * CELLS) < 1.05, (prec, traffic)
        assert 1000 < instr < 10000, (prec, instr)


def test_every_summary_gives_its_command():
    files = sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md")))
    assert files
    for path in files:
        text = open(path).read()
        assert "--clock-control none" in text, path
        assert re.search(r"^\s+(python|ncu) ", text, re.M), path
