"""The kernels' implicit-tree arithmetic (subtree sizes, Sec. 4.1; segment
begin, Sec. 4.2; the position -> subtree inverse that lets the tag be implied
by position) against subtree sizes counted level by level, for every N up to
3000.  Host compile of the same header the CUDA kernels include."""
import os
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_level_layout_against_counted_subtree_sizes(tmp_path):
    exe = str(tmp_path / "index_math_check")
    cuda_inc = "/usr/local/cuda/include"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", cuda_inc, "-I",
                    os.path.join(ROOT, "paper_2211_00120_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "native", "index_math_check.cpp"), "-o", exe],
                   check=True)
    out = subprocess.run([exe, "3000"], capture_output=True, text=True, check=True).stdout
    assert out.startswith("OK"), out
    assert int(out.split()[1]) > 100000
