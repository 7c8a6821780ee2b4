"""The committed ncu records under profiles/ (no GPU needed).

bench.py reports the search kernel's DRAM traffic from the machine-readable
record profiles/search_traffic.json only while that record was taken on the
current search source; a change to the search kernel without a new capture
fails here instead of silently turning the bench's traffic figure to null.
Every ncu command recorded under profiles/ leaves the GPU clocks alone.
"""

import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = os.path.join(ROOT, "profiles")


def test_search_traffic_summary_matches_source():
    import bench
    traffic = bench._profile_traffic()
    assert traffic is not None, "profiles/search_traffic.json was captured on another search source"
    assert traffic > 0


def test_ncu_commands_keep_clocks():
    files = sorted(glob.glob(os.path.join(PROFILES, "*.md")) + glob.glob(os.path.join(PROFILES, "*.txt")))
    assert files
    checked = 0
    for path in files:
        text = open(path).read()
        # join continued shell lines, split chained commands, check each ncu run
        joined = re.sub(r"\\\n\s*", " ", text)
        for line in joined.splitlines():
            for cmd in re.split(r"&&|;|\|", line):
                cmd = cmd.strip()
                if re.match(r"ncu\s", cmd) and not re.search(r"\s-i\s", cmd):
                    checked += 1
                    assert "--clock-control none" in cmd, f"{os.path.basename(path)}: {cmd[:80]}"
    assert checked >= len(files)  # every summary records the capture that made it
