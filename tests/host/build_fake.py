"""Build libhawkes_hosttest.so: the library's host runtime (api.cu as plain C++) linked
against the fake CUDA runtime in fake_cudart.cpp. Test infrastructure only."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "_build", "libhawkes_hosttest.so")
CUDA_INC = os.environ.get("CUDA_INC", "/usr/local/cuda/include")


def build() -> str:
    srcs = [os.path.join(ROOT, "paper_2005_10123_gb300", "csrc", "api.cu"), os.path.join(HERE, "fake_cudart.cpp")]
    deps = srcs + [os.path.join(ROOT, "paper_2005_10123_gb300", "csrc", "hk_internal.h"),
                   os.path.join(ROOT, "paper_2005_10123_gb300", "csrc", "upload.h"),
                   os.path.join(ROOT, "include", "hawkes.h")]
    if os.path.exists(OUT) and all(os.path.getmtime(OUT) >= os.path.getmtime(d) for d in deps):
        return OUT
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    tmp = OUT + f".{os.getpid()}.tmp"
    asan = subprocess.run(["gcc", "-print-file-name=libasan.so"], capture_output=True, text=True).stdout.strip()
    san = ["-fsanitize=address", "-fno-omit-frame-pointer"] if os.path.isabs(asan) and os.path.exists(asan) else []
    cmd = ["g++", "-std=c++17", "-O1", "-g", "-fPIC", "-shared", "-pthread", *san,
           "-I", CUDA_INC, "-I", os.path.join(ROOT, "include"),
           "-x", "c++", srcs[0], "-x", "c++", srcs[1], "-o", tmp]
    subprocess.check_call(cmd)
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build())
