"""Every bench.py command written in profiles/ (the commands that made the
committed ncu summaries) still parses with bench.py's own arguments, so the
summaries stay reproducible from the committed files."""
import glob
import os
import re
import shlex
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench_commands():
    cmds = []
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        text = open(path).read().replace("\\\n", " ")
        for m in re.finditer(r"python bench\.py([^\n`]*)", text):
            cmds.append((os.path.basename(path), shlex.split(m.group(1))))
    return cmds


def test_profile_commands_parse(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    cmds = _bench_commands()
    assert len(cmds) >= 4
    for name, argv in cmds:
        monkeypatch.setattr(sys, "argv", ["bench.py"] + argv)
        args = bench.parse()
        assert args.steps >= 1, name
