"""The FP64 oracle under AddressSanitizer and UndefinedBehaviorSanitizer:
every entry point on small random problems (mode and polarisation-resolved
banks, with and without relative-binning weights, the pre-selection of both,
the weights themselves, the distance marginal and draws), built into one
executable with the sanitizers set to abort on the first report."""
import os
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_oracle_is_clean_under_asan_and_ubsan(tmp_path):
    exe = tmp_path / "oracle_driver"
    cmd = ["gcc", "-O1", "-g", "-std=gnu11", "-pthread", "-fno-omit-frame-pointer", "-fno-fast-math",
           "-fsanitize=address,undefined", "-fno-sanitize-recover=all",
           os.path.join(HERE, "oracle_sanitize_driver.c"), os.path.join(HERE, "..", "oracle", "oracle.c"),
           "-lm", "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip(f"sanitizer build unavailable: {r.stderr[-300:]}")
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0", UBSAN_OPTIONS="print_stacktrace=1")
    r = subprocess.run([str(exe)], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert "runtime error" not in r.stderr and "AddressSanitizer" not in r.stderr, r.stderr[-2000:]
    assert "oracle driver: rc=0" in r.stdout
