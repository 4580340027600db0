"""Every command that a profile summary gives runs committed files only and
passes bench.py's own argument parser."""
import glob
import os
import re
import shlex
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _commands(text):
    # join continuation lines, then keep the "python bench.py ..." parts
    text = re.sub(r"\\\n\s*", " ", text)
    for line in text.splitlines():
        i = line.find("python bench.py")
        if i >= 0:
            cmd = line[i:].split("#")[0].split("`")[0].strip()
            opt = re.search(r"\[(.+?)\]", cmd)  # "[--flag value]": with and without
            if opt:
                yield (cmd[:opt.start()] + cmd[opt.end():]).strip()
                yield (cmd[:opt.start()] + opt.group(1) + cmd[opt.end():]).strip()
            else:
                yield cmd


def test_profile_commands_parse():
    import bench
    seen = 0
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        for cmd in _commands(open(path).read()):
            argv = shlex.split(cmd)[2:]
            # "{a,b,c}" lists alternatives in one line; check each
            alts = [argv]
            for j, a in enumerate(argv):
                m = re.fullmatch(r"\{(.+)\}", a)
                if m:
                    alts = [argv[:j] + [x] + argv[j + 1:] for x in m.group(1).split(",")]
                if a.startswith("<"):
                    alts = [argv[:j] + ["contact"] + argv[j + 1:]]
            for av in alts:
                old = sys.argv
                sys.argv = ["bench.py"] + av
                try:
                    bench.parse()
                finally:
                    sys.argv = old
                seen += 1
    assert seen >= 8
