"""Helpers shared by the tests (build the library, compile the host test executables)."""
import os
import re
import shutil
import subprocess
import tempfile
from concurrent.futures import ThreadPoolExecutor

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qcdmrg.h")


def ensure_built():
    import paper_2603_28648_b300 as qd
    from paper_2603_28648_b300 import build
    if not os.path.exists(qd.LIB_PATH):
        build.build()
    return qd.LIB_PATH


def header_functions():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(qcdmrg_\w+)\s*\(", txt, re.M)))


def cuda_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


CSRC = os.path.join(ROOT, "paper_2603_28648_b300", "csrc")
# the library's host sources that the host test executables link (no CUDA code)
HOST_SOURCES = ["core.cpp", "rules.cpp", "rules_su2.cpp", "su2.cpp", "su2expand.cpp", "init.cpp", "engine.cpp",
                "tiled.cpp"]
_host_objects = {}


def _flags():
    inc = ["-I", CSRC]
    if os.path.isdir("/usr/local/cuda/include"):
        inc += ["-I", "/usr/local/cuda/include"]
    return ["-O2", "-std=c++17", "-pthread"] + inc


def host_objects():
    """The host sources compiled once per test session, in parallel; object paths."""
    if "objs" not in _host_objects:
        d = tempfile.mkdtemp(prefix="qcdmrg_host_")
        objs = [os.path.join(d, s.replace(".cpp", ".o")) for s in HOST_SOURCES]

        def one(args):
            src, obj = args
            subprocess.run(["g++"] + _flags() + ["-c", os.path.join(CSRC, src), "-o", obj], check=True)

        with ThreadPoolExecutor(max_workers=min(len(objs), os.cpu_count() or 1)) as pool:
            list(pool.map(one, zip(HOST_SOURCES, objs)))
        _host_objects["objs"] = objs
    return _host_objects["objs"]


def build_host_executable(main_cpp, out):
    """tests/<main_cpp> linked with the library's host sources into out (None without g++)."""
    if shutil.which("g++") is None:
        return None
    subprocess.run(["g++"] + _flags() + [os.path.join(ROOT, "tests", main_cpp)] + host_objects() + ["-o", out],
                   check=True)
    return out
