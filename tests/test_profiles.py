"""The ncu summaries under profiles/: each names the command that made it
(run from the repository root on committed files, with the clocks left as
they were), and each kernel capture records the source file and sha256 of
the kernel it measured plus the DRAM counters bench.py reads (no GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROF = os.path.join(ROOT, "profiles")
FILES = sorted(f for f in os.listdir(PROF) if f.endswith(".md"))


def test_there_are_summaries():
    assert any(f.startswith("launches_") for f in FILES)
    assert sum(f.startswith("k_") for f in FILES) >= 5


@pytest.mark.parametrize("name", FILES)
def test_summary_is_well_formed(name):
    text = open(os.path.join(PROF, name)).read()
    cmds = re.findall(r"```\n(.*?)\n```", text, re.S)
    assert cmds, "no command block"
    cmd = cmds[0]
    assert "ncu " in cmd and "--clock-control none" in cmd
    # the profiled program is one of the repository's own entry points
    prog = re.search(r"(python (?:-m pytest )?\S+)", cmd.split("ncu ", 1)[1])
    assert prog, cmd
    target = prog.group(1).split()[-1]
    assert os.path.exists(os.path.join(ROOT, target)), target
    assert "_work" not in cmd and "/root" not in cmd
    if name.startswith("k_"):
        m = re.search(r"Kernel source at capture: `([^`]+)` sha256 ([0-9a-f]{16})",
                      text)
        assert m and os.path.exists(os.path.join(ROOT, m.group(1)))
        for metric in ("gpu__time_duration.sum", "dram__bytes_read.sum",
                       "dram__bytes_write.sum"):
            assert re.search(r"`%s` \| [0-9.]+ \w+" % re.escape(metric), text), metric
        assert re.search(r"Algorithmic bytes of the captured launch: \d+", text)
