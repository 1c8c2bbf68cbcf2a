"""Repository rules that keep the measurements reproducible: every profile summary gives the
ncu command that made it, each with --clock-control none, and runs committed files only; no
committed file refers to the untracked scratch folder."""
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _tracked():
    out = subprocess.run(["git", "ls-files"], capture_output=True, text=True, cwd=ROOT)
    return [f for f in out.stdout.splitlines() if f]


def test_profile_summaries_carry_their_commands():
    prof = os.path.join(ROOT, "profiles")
    names = [f for f in os.listdir(prof) if f.endswith(".md")]
    assert names
    for f in names:
        text = open(os.path.join(prof, f)).read()
        cmds = [ln for ln in text.splitlines() if re.match(r"\s*ncu\s", ln)]
        assert cmds, f
        assert all("--clock-control none" in c for c in cmds), f


def test_no_committed_file_uses_the_scratch_folder():
    files = _tracked()
    if not files:          # not a git checkout (e.g. a copy without .git)
        return
    scratch = "_" + "work/"
    for f in files:
        if f.endswith((".md", ".txt", ".py", ".cu", ".cuh", ".h", ".c", ".json")) and \
                f != ".gitignore":
            with open(os.path.join(ROOT, f), errors="replace") as fh:
                assert scratch not in fh.read(), f
