"""The committed profiler summaries (profiles/*.md), checked on the CPU: each
gives the commands that made it, and those commands must run committed
files only, with flags the benchmark accepts, and every ncu capture must
leave the GPU clocks alone (--clock-control none) and, when it collects more
than the launch list, name one kernel (-k) and a launch count (-c)."""
import glob
import os
import re
import shlex

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md")))


def _commands(path):
    """Shell commands in a summary: lines that start (after indentation or
    a code fence) with python or ncu, joined across trailing backslashes."""
    cmds, cur = [], None
    for raw in open(path):
        line = raw.rstrip("\n")
        body = line.split("#", 1)[0].rstrip() if not line.lstrip().startswith("#") else ""
        if cur is not None:
            cur += " " + body.rstrip("\\").strip()
            if not body.endswith("\\"):
                cmds.append(cur)
                cur = None
            continue
        s = body.strip()
        if s.startswith("python ") or s.startswith("ncu ") or s.startswith("<cmd>"):
            if s.endswith("\\"):
                cur = s.rstrip("\\").strip()
            else:
                cmds.append(s)
    if cur is not None:
        cmds.append(cur)
    return cmds


def _bench_flags():
    src = open(os.path.join(ROOT, "bench.py")).read()
    flags = set(re.findall(r'add_argument\("(--[a-z0-9-]+)"', src))
    m = re.search(r'"--only", choices=\[([^\]]*)\]', src, re.S)
    only = set(re.findall(r'"([a-z0-9-]+)"', m.group(1)))
    return flags, only


def test_every_summary_gives_its_commands():
    assert PROFILES
    for p in PROFILES:
        assert _commands(p), f"{os.path.basename(p)} gives no command"


def test_ncu_commands_leave_the_clocks_alone_and_stay_small():
    for p in PROFILES:
        for c in _commands(p):
            if not c.startswith("ncu "):
                continue
            assert "--clock-control none" in c, (os.path.basename(p), c)
            if "--set" in c or "--section" in c:
                assert re.search(r"(^|\s)-k\s", c) and re.search(r"(^|\s)-c\s", c), (os.path.basename(p), c)


def test_commands_run_committed_files_with_flags_the_benchmark_accepts():
    flags, only = _bench_flags()
    for p in PROFILES:
        for c in _commands(p):
            assert "_work/" not in c, (os.path.basename(p), c)
            toks = shlex.split(c.replace("&&", " "))
            if "bench.py" not in toks:
                continue
            args = toks[toks.index("bench.py") + 1:]
            for i, t in enumerate(args):
                if t.startswith("--"):
                    assert t.split("=", 1)[0] in flags, (os.path.basename(p), t)
                    if t == "--only":
                        assert args[i + 1] in only, (os.path.basename(p), args[i + 1])
