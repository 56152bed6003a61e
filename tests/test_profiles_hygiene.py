"""The committed ncu summaries under profiles/: short text files named for a
kernel (or launch list) and workload, each giving the full command that made
it, and every ncu command in them leaves the GPU clocks alone
(--clock-control none)."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROF = os.path.join(ROOT, "profiles")


def _commands(text):
    """shell commands of the summary, backslash continuations joined"""
    joined = re.sub(r"\\\n\s*", " ", text)
    return [ln.strip() for ln in joined.splitlines() if re.search(r"(^|&&)\s*ncu\s+-", ln.strip())]


def test_profiles_are_short_text_named_for_kernel_and_workload():
    names = sorted(os.listdir(PROF))
    assert names
    for n in names:
        assert n.endswith((".md", ".txt")), n
        assert os.path.getsize(os.path.join(PROF, n)) < 16 * 1024, n
        assert n.startswith(("k_", "launches_", "roofline_")), n
        assert not re.search(r"(^|_)r\d\d|round", n), n


def test_every_ncu_command_keeps_the_clocks():
    seen = 0
    for n in sorted(os.listdir(PROF)):
        text = open(os.path.join(PROF, n)).read()
        cmds = _commands(text)
        assert cmds, f"{n}: no ncu command given"
        for c in cmds:
            seen += 1
            assert "--clock-control none" in c, (n, c)
    assert seen > 0
