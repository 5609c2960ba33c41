"""The CPU oracle under AddressSanitizer and UndefinedBehaviorSanitizer: a C
driver (tests/host/oracle_sanitize.c) calls every oracle entry point on small
random inputs; any memory error, leak or undefined behaviour aborts it."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_oracle_is_clean_under_asan_and_ubsan():
    if shutil.which("gcc") is None:
        pytest.skip("needs gcc")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "oracle_sanitize")
        cmd = ["gcc", "-std=c11", "-O1", "-g", "-ffp-contract=off", "-fno-fast-math",
               "-fsanitize=address,undefined", "-fno-sanitize-recover=all", "-fno-omit-frame-pointer",
               "-I", os.path.join(ROOT, "oracle"), os.path.join(ROOT, "tests", "host", "oracle_sanitize.c"),
               os.path.join(ROOT, "oracle", "rawalign_oracle.c"), "-lm", "-o", exe]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0 and "sanitize" in (r.stderr or ""):
            pytest.skip("compiler without sanitizer runtime: " + r.stderr[-300:])
        assert r.returncode == 0, r.stderr[-3000:]
        env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=1",
                   UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1")
        out = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=600)
        assert out.returncode == 0, (out.stdout + out.stderr)[-4000:]
        assert "no report" in out.stdout
