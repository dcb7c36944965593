"""The ncu summaries under profiles/ name commands that run committed files:
every bench.py invocation they quote parses with bench.py's own argument
parser, and every traffic entry the bench reads names a summary that exists."""
import json
import os
import re
import shlex

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = os.path.join(ROOT, "profiles")


def _bench_invocations():
    out = []
    for name in sorted(os.listdir(PROFILES)):
        if not name.endswith(".md"):
            continue
        with open(os.path.join(PROFILES, name)) as f:
            text = f.read().replace("\\\n", " ")
        for m in re.finditer(r"python bench\.py([^\n>`&]*)", text):
            out.append((name, m.group(1)))
    return out


def test_profile_commands_parse():
    import bench
    calls = _bench_invocations()
    assert calls, "no bench.py command found in profiles/"
    ap = bench.make_parser()
    for name, argstr in calls:
        args = ap.parse_args(shlex.split(argstr))      # exits (fails the test) on an unknown flag or case
        assert args is not None, name


def test_every_profile_names_its_command():
    for name in os.listdir(PROFILES):
        if name.endswith(".md"):
            with open(os.path.join(PROFILES, name)) as f:
                text = f.read()
            assert "ncu " in text and "--clock-control none" in text, name


def test_traffic_sources_exist():
    with open(os.path.join(PROFILES, "traffic.json")) as f:
        traffic = json.load(f)
    for kernel, entries in traffic.items():
        for e in entries if isinstance(entries, list) else [entries]:
            src = e["source"].split(":")[0]
            assert os.path.exists(os.path.join(ROOT, src)), (kernel, src)
            assert e["bytes_per_flop"] > 0 and e["k"] > 0
