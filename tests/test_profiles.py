"""The ncu summaries under profiles/: each states the command that made it,
with the clock control left to the GPU (--clock-control none), running
files of this repository only."""

import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _commands(text):
    # indented command blocks, continuation lines joined
    out, cur = [], []
    for line in text.splitlines():
        if line.startswith("    ") and line.strip():
            cur.append(line.strip().rstrip("\\").strip())
            if not line.rstrip().endswith("\\"):
                out.append(" ".join(cur))
                cur = []
    return out


def test_every_summary_names_its_command():
    files = sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md")))
    assert files
    for path in files:
        cmds = [c for c in _commands(open(path).read()) if c.startswith("ncu ")]
        assert cmds, path
        for c in cmds:
            assert "--clock-control none" in c, (path, c)
            scripts = re.findall(r"python (?:-m )?(\S+)", c)
            assert scripts, (path, c)
            for s in scripts:
                if s.endswith(".py"):
                    assert os.path.exists(os.path.join(ROOT, s)), (path, s)
                else:   # a module of this repository
                    rel = s.replace(".", os.sep)
                    assert (os.path.exists(os.path.join(ROOT, rel + ".py"))
                            or os.path.isdir(os.path.join(ROOT, rel))), (path, s)
