"""The ncu summaries under profiles/: short text files, each giving the command that made
it, with the clocks left alone (--clock-control none), running a committed script whose
arguments that script still accepts."""
import glob
import os
import re
import shlex
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = sorted(glob.glob(os.path.join(ROOT, "profiles", "*")))


def _commands(text):
    """ncu command lines of a summary, backslash continuations joined."""
    joined = re.sub(r"\\\n\s*", " ", text)
    return [ln.strip() for ln in joined.splitlines() if ln.strip().startswith("ncu ")]


def test_profiles_are_short_text():
    assert PROFILES
    for p in PROFILES:
        assert p.endswith((".md", ".txt")), p
        assert os.path.getsize(p) < 16 * 1024, p


@pytest.mark.parametrize("path", PROFILES, ids=os.path.basename)
def test_profile_command_runs_committed_code(path, monkeypatch):
    cmds = _commands(open(path).read())
    assert cmds, f"{path}: no ncu command"
    sys.path.insert(0, ROOT)
    import bench

    for cmd in cmds:
        assert "--clock-control none" in cmd, cmd
        words = shlex.split(cmd)
        k = words.index("python")
        script, args = words[k + 1], words[k + 2:]
        assert os.path.exists(os.path.join(ROOT, script)), script
        assert script == "bench.py", script
        monkeypatch.setattr(sys, "argv", ["bench.py", *args])
        bench.parse_args()  # exits (SystemExit) on an argument the script no longer takes
