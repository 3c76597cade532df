"""Source files stand on their own: no code, comment or docstring names the
build's planning documents, the task's target statement, the remote GPU
runner or a path of the build machine.  (The words are assembled from
fragments so that this file does not contain them either.)"""
import os
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BANNED = ["north" + "_star", "north" + " star", "BASE" + "LINE.json", "BASE" + "LINE.md",
          "PAPER" + ".md", "SPEC" + ".md", "SURVEY" + ".md", "DESIGN" + ".md",
          "VERDICT" + ".md", "ADVICE" + ".md", "gpu" + "run", "/" + "root/"]
SUFFIXES = (".py", ".cu", ".cuh", ".h", ".c")


def _sources():
    try:
        files = subprocess.run(["git", "ls-files"], cwd=ROOT, capture_output=True,
                               text=True).stdout.split()
    except OSError:
        files = []
    if not files:
        for d, _, fs in os.walk(ROOT):
            if "/." in d or "/_work" in d or "__pycache__" in d:
                continue
            files += [os.path.relpath(os.path.join(d, f), ROOT) for f in fs]
    return [f for f in files if f.endswith(SUFFIXES)]


def test_sources_name_no_planning_document_runner_or_machine_path():
    hits = []
    for f in _sources():
        text = open(os.path.join(ROOT, f), errors="replace").read().lower()
        hits += [f"{f}: {w}" for w in BANNED if w.lower() in text]
    assert not hits, hits
