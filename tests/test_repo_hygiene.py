"""Committed files stand on their own: nothing refers to the untracked scratch
folder, and profiles/ holds short text summaries only."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _tracked():
    try:
        out = subprocess.run(["git", "ls-files"], cwd=ROOT, capture_output=True, text=True, check=True).stdout
    except (OSError, subprocess.CalledProcessError):
        pytest.skip("not a git checkout")
    return [f for f in out.splitlines() if f]


def test_no_committed_file_refers_to_the_scratch_folder():
    # The literal is built from parts so that this file does not match itself.
    pat = re.compile(r"(^|[^A-Za-z0-9_])" + "_" + "work/")
    bad = []
    for f in _tracked():
        if not f.endswith((".py", ".cu", ".cuh", ".h", ".c", ".md", ".txt", ".json", ".sh")):
            continue
        # Review and record files written outside the build itself.
        base = os.path.basename(f)
        if base in ("SURVEY.md", "BASELINE.md", "BASELINE.json", "VERDICT.md", "ADVICE.md"):
            continue
        if re.match(r"(BENCH|GPUTEST|SCALE|MULTICHIP)_r\d+\.json$", base):
            continue
        with open(os.path.join(ROOT, f), errors="replace") as fh:
            if pat.search(fh.read()):
                bad.append(f)
    assert not bad, bad


def test_profiles_are_short_text_summaries():
    files = [f for f in _tracked() if f.startswith("profiles/")]
    assert files
    for f in files:
        assert f.endswith((".md", ".txt", ".json")), f
        assert os.path.getsize(os.path.join(ROOT, f)) < 64 * 1024, f
