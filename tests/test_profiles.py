"""The committed ncu summaries: each names the command that made it, and that command runs committed files only
(no scratch paths), so that anyone can take the capture again."""
import glob
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _tracked():
    out = subprocess.run(["git", "ls-files"], cwd=ROOT, capture_output=True, text=True)
    return set(out.stdout.split()) if out.returncode == 0 else None


def test_every_summary_gives_its_command_and_runs_committed_files_only():
    summaries = sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md")))
    assert summaries
    tracked = _tracked()
    for path in summaries:
        text = open(path).read()
        name = os.path.basename(path)
        assert re.search(r"\b(ncu|python)\b", text), f"{name}: no command"
        assert "_work" not in text, f"{name}: names a scratch path"
        for script in re.findall(r"python\s+(?!-m\b)([\w./-]+\.py)", text):
            assert os.path.exists(os.path.join(ROOT, script)), f"{name}: {script} does not exist"
            if tracked is not None:
                assert script in tracked, f"{name}: {script} is not committed"
