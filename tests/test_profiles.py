"""The committed ncu summaries (CPU, static): each names the command that made it, every ncu
invocation leaves the GPU clocks alone (--clock-control none), and the profiled program is
bench.py with one of its own --profile modes, a committed file and nothing else."""
import glob
import os
import re

from tests.conftest import ROOT


def _commands(text):
    """The shell commands of a summary's code blocks, continuation lines joined."""
    out = []
    for block in re.findall(r"```[a-z]*\n(.*?)```", text, re.S):
        joined = re.sub(r"\\\n\s*", " ", block)
        out.extend(c.strip() for line in joined.splitlines() for c in line.split("&&") if c.strip())
    return out


def test_every_summary_names_its_command():
    modes = {m.strip().strip('"') for m in re.search(r'"--profile", choices=\[([^\]]*)\]',
                                                      open(os.path.join(ROOT, "bench.py")).read()).group(1).split(",")}
    paths = sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md")))
    assert paths
    for path in paths:
        cmds = _commands(open(path).read())
        ncu = [c for c in cmds if c.startswith("ncu ")]
        assert ncu, f"{os.path.basename(path)}: no ncu command"
        for c in ncu:
            assert "--clock-control none" in c, f"{os.path.basename(path)}: {c}"
        for c in cmds:
            if c.startswith(("ncu ", "python ")):
                prog = re.search(r"python (\S+)(.*)$", c)
                assert prog and prog.group(1) == "bench.py", f"{os.path.basename(path)}: {c}"
                mode = re.search(r"--profile (\w+)", prog.group(2))
                assert mode and mode.group(1) in modes, f"{os.path.basename(path)}: {c}"
