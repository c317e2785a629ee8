"""Helpers shared by the tests (build the library, oracle-side MPS export)."""
import os
import re

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
