"""The CPU oracle and the parallel CPU port under AddressSanitizer and
UndefinedBehaviorSanitizer (host only): a C driver builds, checks and
cross-checks them over edge sizes, split rules, coordinate types, payload
strides, ties, extremes, NaN and bad arguments, and any out-of-bounds access,
leak or undefined operation (signed overflow, bad shift) aborts the run."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SAN = ["-fsanitize=address,undefined", "-fno-sanitize-recover=all", "-fno-omit-frame-pointer"]


def _sanitizers_available(tmp_path):
    src = tmp_path / "probe.c"
    src.write_text("int main(void) { return 0; }\n")
    r = subprocess.run(["gcc", *SAN, str(src), "-o", str(tmp_path / "probe")], capture_output=True)
    return r.returncode == 0


def test_oracle_and_cpu_port_are_clean_under_sanitizers(tmp_path):
    if not _sanitizers_available(tmp_path):
        pytest.skip("gcc sanitizer runtimes are not installed")
    exe = str(tmp_path / "oracle_sanitize")
    subprocess.run(["gcc", "-O1", "-g", "-std=c11", *SAN,
                    os.path.join(ROOT, "tests", "native", "oracle_sanitize.c"),
                    os.path.join(ROOT, "oracle", "kd_oracle.c"),
                    os.path.join(ROOT, "oracle", "paper_cpu.c"),
                    "-o", exe, "-lpthread", "-lm"], check=True)
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=1",
               UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1")
    r = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, (r.stdout[-2000:], r.stderr[-4000:])
    assert r.stdout.startswith("OK"), r.stdout[-2000:]
    assert int(r.stdout.split()[1]) > 40000
