"""The bench's roofline model restates two constants of the scan kernels:
the window-sliced cut (ws_cut, list entries tested before the remaining
candidates are counted one by one) and the tile widths.  The kernels'
own definitions, compiled for the host by nvcc, must agree with it."""
import os
import shutil
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1611_06115_gb300", "csrc")

PROBE = r"""
#include <cstdio>
#include "pm_scan_impl.cuh"
int main()
{
    for (int k = 0; k <= pm::kWsMaxK; ++k) std::printf("%u ", pm::scan::ws_cut(k));
    std::printf("\n%d %d\n", pm::scan_groups(pm::Variant::kWindowSliced, 4),
                pm::scan_groups(pm::Variant::kPatternSliced, 16));
    return 0;
}
"""


def test_ws_cut_and_tile_widths_match_the_kernels(tmp_path):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not found")
    src = tmp_path / "probe.cu"
    src.write_text(PROBE)
    exe = str(tmp_path / "probe")
    r = subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include"),
                        "-I", CSRC, str(src), "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    cuts = [int(x) for x in out[0].split()]
    sys.path.insert(0, ROOT)
    import bench
    assert cuts == [bench.ws_cut(k) for k in range(len(cuts))]
    ws_groups, ps_groups = (int(x) for x in out[1].split())
    assert (ws_groups, ps_groups) == (8, 4)
