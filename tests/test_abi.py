"""The CUDA library builds, loads, and exports every entry point include/hawkes.h declares
(no compute calls: this runs without a GPU)."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "hawkes.h")) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hawkes_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("hawkes_upload_events", "hawkes_loglik", "hawkes_loglik_grad", "hawkes_submit",
                     "hawkes_poll", "hawkes_wait"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2005_10123_gb300 import binding, build
    build.build()
    lib = binding.load()
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(_declared()) == set(binding.EXPORTS)


def test_library_fails_cleanly_without_gpu():
    """Without a usable device, context creation returns a status code (no abort)."""
    import ctypes
    import torch
    if torch.cuda.is_available():
        return
    from paper_2005_10123_gb300 import binding
    lib = binding.load()
    h = ctypes.c_void_p()
    rc = lib.hawkes_create(ctypes.byref(h), 0, 0, None)
    assert rc != 0
    assert lib.hawkes_strerror(rc)
