"""Every profile summary names the commands that produced its figures, and
those commands run files of this repository only."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = os.path.join(ROOT, "profiles")


def summaries():
    return sorted(f for f in os.listdir(PROFILES) if f.endswith(".md"))


@pytest.mark.parametrize("name", summaries())
def test_profile_commands_run_committed_files(name):
    text = open(os.path.join(PROFILES, name)).read()
    scripts = re.findall(r"python3? (?!-m)([\w./-]+\.py)", text)
    modules = re.findall(r"python3? -m ([\w.]+)", text)
    assert scripts or modules, f"{name} names no command"
    for s in scripts:
        assert os.path.exists(os.path.join(ROOT, s)), (name, s)
    for m in modules:
        path = os.path.join(ROOT, *m.split("."))
        assert os.path.exists(path + ".py") or os.path.isdir(path), (name, m)
    assert "_work" not in text, name
