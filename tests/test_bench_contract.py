"""Host-side pieces of bench.py that need no GPU: the launch count's queue classes follow the
library's rule (wos_launch.h), and the DRAM traffic of a committed ncu summary is reported only
while the kernel sources hash to the recorded value."""
import os
import re
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

LAUNCH_H = os.path.join(ROOT, "paper_2406_01713_gb300", "csrc", "wos_launch.h")


def header_constant(name):
    m = re.search(r"constexpr int %s = (\d+);" % name, open(LAUNCH_H).read())
    assert m, name
    return int(m.group(1))


def test_queue_classes_follow_the_library():
    wide_tiles = header_constant("kSphereWideTiles")
    wide_max_d = header_constant("kSphereWideMaxD")
    large_tiles = header_constant("kSphereLargeTiles")
    for d in range(2, 13):
        for tiles in range(1, 400):
            want = 2 if (d <= wide_max_d and tiles >= wide_tiles) else (1 if tiles >= large_tiles else 0)
            assert bench.sphere_queue_class(d, tiles) == want, (d, tiles)


@pytest.mark.parametrize("profile,sources", [(bench.TRAFFIC_PROFILE, bench.KERNEL_SOURCES),
                                             (bench.SPHERE_TRAFFIC_PROFILE, bench.SPHERE_SOURCES)])
def test_traffic_only_for_the_recorded_sources(profile, sources):
    vals = {}
    for line in open(os.path.join(ROOT, profile)):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            vals[k] = v
    got = bench.measured_traffic(profile, sources)
    assert got == int(vals["dram_bytes_read"]) + int(vals["dram_bytes_write"])
    # a different source list no longer hashes to the recorded value
    assert bench.measured_traffic(profile, sources[1:]) is None
