"""Host logic of the library (uploads, schedules, batching, serving queue, admission,
allocation faults, timeouts) on the CPU, against a fake CUDA runtime. The checks run in
a subprocess under AddressSanitizer when the compiler ships it."""
import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _asan_runtime():
    try:
        p = subprocess.run(["gcc", "-print-file-name=libasan.so"], capture_output=True, text=True).stdout.strip()
    except OSError:
        return None
    return p if p and os.path.isabs(p) and os.path.exists(p) else None


def test_host_runtime_checks():
    sys.path.insert(0, os.path.join(HERE, "host"))
    try:
        import build_fake
    finally:
        sys.path.pop(0)
    try:
        build_fake.build()
    except OSError as e:  # no host compiler: nothing to test with
        pytest.skip(f"cannot run the host compiler: {e}")
    except subprocess.CalledProcessError as e:  # the library's host code no longer compiles
        pytest.fail(f"the host-test library does not build: {e}")
    env = dict(os.environ)
    asan = _asan_runtime()
    if asan:
        env["LD_PRELOAD"] = asan
        env["ASAN_OPTIONS"] = "detect_leaks=0:abort_on_error=1"
    # uploads both ways: a copy of the caller's arrays, and a device that reads them in place
    for direct in ("0", "1"):
        env["FAKE_HOST_DIRECT"] = direct
        r = subprocess.run([sys.executable, os.path.join(HERE, "host", "host_checks.py")], env=env,
                           capture_output=True, text=True, timeout=600)
        assert r.returncode == 0 and "ALL OK" in r.stdout, r.stdout[-3000:] + r.stderr[-6000:]
