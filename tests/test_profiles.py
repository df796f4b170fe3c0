"""Every ncu summary under profiles/ gives the command that made it; those
commands must still run against the committed bench.py (its argument
parser accepts them) and name only committed files."""
import glob
import os
import re
import shlex
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def quoted_commands():
    out = []
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        text = open(path).read().replace("\\\n", " ")
        for raw in text.splitlines():
            line = raw.strip()
            # commands sit in indented code blocks
            if raw.startswith("    ") and (line.startswith("ncu ") or line.startswith("python bench.py")):
                out.append((os.path.basename(path), line))
    return out


def test_each_summary_quotes_its_command():
    names = {name for name, _ in quoted_commands()}
    for path in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        assert os.path.basename(path) in names, path


def test_quoted_commands_parse_against_bench():
    sys.path.insert(0, ROOT)
    import bench
    for name, cmd in quoted_commands():
        words = shlex.split(cmd)
        assert "bench.py" in words, (name, cmd)
        if words[0] == "ncu":
            assert "--clock-control" in words and words[words.index("--clock-control") + 1] == "none", name
        args = words[words.index("bench.py") + 1:]
        saved = sys.argv
        try:
            sys.argv = ["bench.py", *args]
            a = bench.args_()
        finally:
            sys.argv = saved
        assert a.impl == "ours", (name, cmd)
        assert re.fullmatch(r"python", words[words.index("bench.py") - 1]), (name, cmd)
