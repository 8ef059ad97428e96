"""The library's host-side code under AddressSanitizer and
UndefinedBehaviorSanitizer: the CUDA sources compiled with sanitized host
code and linked into a C++ driver that exercises build plans (single and
batched workspace layouts over many sizes, dimensions, strides and modes),
the tile-shape setting and the tuning-file parser on random input.  No GPU
call is made."""
import concurrent.futures as cf
import os
import shutil
import subprocess

import pytest

from paper_2211_00120_gb300 import build_lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SAN = ["-fsanitize=address", "-fsanitize=undefined", "-fno-sanitize-recover=all",
       "-fno-omit-frame-pointer"]


def test_host_code_is_clean_under_sanitizers(tmp_path):
    probe = tmp_path / "probe.cpp"
    probe.write_text("int main() { return 0; }\n")
    if subprocess.run(["g++", *SAN, str(probe), "-o", str(tmp_path / "probe")],
                      capture_output=True).returncode != 0:
        pytest.skip("gcc sanitizer runtimes are not installed")
    nvcc = build_lib.nvcc()
    cuda_lib = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "lib64")
    if not os.path.exists(os.path.join(cuda_lib, "libcudart_static.a")):
        pytest.skip("static CUDA runtime not found")

    def compile_one(src):
        obj = str(tmp_path / (os.path.splitext(src)[0] + ".o"))
        cmd = [nvcc, "-c", os.path.join(build_lib.CSRC, src), "-o", obj] + build_lib.ARCH + \
              ["-O1", "-std=c++17", "-I", os.path.join(ROOT, "include"), "--expt-relaxed-constexpr"]
        for f in SAN:
            cmd += ["-Xcompiler", f]
        subprocess.run(cmd, check=True, capture_output=True)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(build_lib.SOURCES)) as ex:
        objs = list(ex.map(compile_one, build_lib.SOURCES))
    exe = str(tmp_path / "host_plan_sanitize")
    subprocess.run([shutil.which("g++") or "g++", "-O1", "-g", "-std=c++17", *SAN, "-I",
                    os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "native", "host_plan_sanitize.cpp"), *objs,
                    "-L", cuda_lib, "-lcudart_static", "-ldl", "-lpthread", "-lrt", "-o", exe],
                   check=True)
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:protect_shadow_gap=0:abort_on_error=1",
               UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1")
    r = subprocess.run([exe, str(tmp_path / "tuning.json")], capture_output=True, text=True,
                       env=env, timeout=300)
    assert r.returncode == 0, (r.stdout[-2000:], r.stderr[-4000:])
    assert r.stdout.startswith("OK"), r.stdout[-2000:]
    assert int(r.stdout.split()[1]) > 10000
